// Dense pieces of the preconditioners (sm_103a):
//   * k_dense_prep / k_gram_gemm / k_gram_tiles / k_gram_diag_hs : K = Hs + R^T diag(omega) R +
//                  U W U^T + diag(h0 + sigma), scaled by a power of two, as a dense n x n
//                  matrix (the DENSE preconditioner: one diagonal block covering all variables);
//   * k_chol_*   : in-place blocked Cholesky factor (lower) with pivot flooring, and the
//                  reciprocal pivots;
//   * k_chol_tile_inv : inverses of the factor's 32 x 32 diagonal tiles;
//   * k_mirror   : last pass of a factorisation: installs the factored diagonal tiles and copies
//                  L^T into the upper triangle, so both triangular sweeps read rows;
//   * k_inv      : explicit inverse from the factor, columns spread over blocks.
// The low-rank correction's G (up to 1024 rows) is factored in float64 and inverted
// explicitly, so each of the many PCG applies is a parallel matvec.  The DENSE
// preconditioner, whose PCG takes one or two iterations, is formed, factored and applied
// (triangular solves, k_dense_trsv) in double-float arithmetic: values are pairs of float32
// (hi + lo, about 48 bits) computed on the float32 pipe.  On GB300 a dependent float64
// multiply-add takes 64 cycles, a float64 rsqrt or division over 400, and the SM retires one
// float64 warp instruction per ~19 cycles, against 4.5 cycles and 128 lanes per clock for
// float32: the factorisation is a chain of dependent steps and the Gram product is bound by
// arithmetic, so both run several times faster in pairs.  A preconditioner needs no more than
// the pairs' precision; PCG on the float64 operator carries the solve to its tolerance.
// Pairs keep float32's exponent range, so K is scaled by 2^-2e (exact, e chosen each IPM
// iteration from float64 bounds on its entries) before it is formed; the solve undoes it.
// The factorisation runs once per IPM iteration.
#include <algorithm>
#include <cmath>

#include "state.h"

namespace ipmk {

// ------------------------------------------------------------------ scalar policies
// float64 (the stiff-row G) and double-float pairs in a float2 (x + y, |y| <= ulp(x) / 2
// after each operation; the dense K).

__device__ __forceinline__ double r_mul(double a, double b) { return a * b; }
__device__ __forceinline__ double r_fms(double c, double a, double b) { return fma(-a, b, c); }   // c - a b
__device__ __forceinline__ double r_rsqrt(double p) { return rsqrt(p); }
__device__ __forceinline__ bool r_above(double a, double b) { return a > b; }
__device__ __forceinline__ double r_shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double r_to_double(double v) { return v; }
__device__ __forceinline__ double r_floor(double fl) { return fl + 1e-300; }
template <class R> __device__ __forceinline__ R r_const(double v);
template <> __device__ __forceinline__ double r_const<double>(double v) { return v; }
template <> __device__ __forceinline__ float2 r_const<float2>(double v) { return make_float2((float)v, 0.f); }

// a b: the high product, its exact error (fma) and the two cross terms
__device__ __forceinline__ float2 r_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return df_fast_sum(p, e);
}
// c - a b
__device__ __forceinline__ float2 r_fms(float2 c, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  float s, t;
  two_sum(c.x, -p, s, t);
  t = __fadd_rn(t, __fsub_rn(c.y, e));
  return df_fast_sum(s, t);
}
// 1 / sqrt(p): the float32 estimate r0, then one Newton step r0 + r0 (1 - p r0^2) / 2 with
// the residual 1 - p r0^2 formed in pairs (r0^2 exact by fma)
__device__ __forceinline__ float2 r_rsqrt(float2 p) {
  const float r0 = rsqrtf(p.x);
  const float q = __fmul_rn(r0, r0);
  const float2 w = r_mul(p, make_float2(q, __fmaf_rn(r0, r0, -q)));
  const float e = __fsub_rn(__fsub_rn(1.f, w.x), w.y);
  return df_fast_sum(r0, __fmul_rn(__fmul_rn(0.5f, r0), e));
}
__device__ __forceinline__ bool r_above(float2 a, float2 b) { return a.x > b.x; }
__device__ __forceinline__ float2 r_shfl(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ double r_to_double(float2 v) { return df_value(v.x, v.y); }
__device__ __forceinline__ float2 r_floor(float2 fl) { return make_float2(fmaxf(fl.x, 1e-30f), 0.f); }

// ------------------------------------------------------------------ blocked Cholesky
// Blocked right-looking Cholesky (lower, row-major, leading dimension ld) of the leading
// nn x nn block of A on 32 x 32 tiles, two launches per tile column kb:
//   * the panel: every block factors the diagonal tile in shared memory (the same code on the
//     same data, so each gets the same factor; block 0 stores it in tiles[kb], which the last
//     pass installs), then the others each solve 16 rows of the tiles below,
//     X = A_ib,kb L_kb,kb^{-T}, one warp per row;
//   * the trailing update A_ib,jb -= L_ib,kb L_jb,kb^T (kb < jb <= ib) on 16 x 16 quarter tiles.
// Each pivot takes one reciprocal square root and the rest multiplies by it (no division on
// the chain), and the arithmetic of a tile column is spread over as many SMs as it has row
// blocks.  The reciprocal pivots go to rinv[] for the triangular solves.  nn is read on the
// device (it may be the number of stiff rows).  A pivot below floor_rel * (original diagonal)
// is raised to that floor (a modified factor; still symmetric positive definite, which is all
// a preconditioner needs); the count goes to *nfloor.
constexpr int kT = 32;
constexpr int kPanelRows = 16;  // rows of the panel below the diagonal tile per block (a warp each)
constexpr double kFloorRel = 1e-13;

__device__ __forceinline__ int dev_nn(const int* nn_dev, int nn_fixed) { return nn_dev ? *nn_dev : nn_fixed; }

template <class R>
__global__ void k_chol_save_diag(const R* A, int64_t ld, const int* nn_dev, int nn_fixed, double* diag0, int* nfloor) {
  const int nn = dev_nn(nn_dev, nn_fixed);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x)
    diag0[i] = r_to_double(A[(int64_t)i * ld + i]);
  if (blockIdx.x == 0 && threadIdx.x == 0 && nfloor) *nfloor = 0;
}

// Unblocked Cholesky of diagonal tile kb in shared memory (rows/cols >= nn padded by
// identity): rs[k] = 1 / L_kk.  Pivots are floored as above; nfloor (may be null) counts the
// floored ones.  The pivots form a chain, so each step is organised around it with one
// barrier: warp 0 holds column k in registers (lane i: L_ik), applies step k to column k + 1
// and factors it at once (pivot by shuffle, reciprocal square root, scaling), while the
// other warps apply step k to the rest of the trailing block, the entries (i, j) with
// k + 1 < j <= i.  Listed by j descending (then i), those are the first (30 - k)(31 - k) / 2
// entries of one table of pairs, so the threads take them densely (one each with 512
// threads) instead of one row per warp with most lanes idle.  (Measured on GB300: about
// 20000 cycles per tile; a whole tile in one warp's registers, with no barrier, took 44000:
// one warp then issues every multiply-add of the tile.)
constexpr int kPanelThreads = 512;
constexpr int kTriPairs = kT * (kT - 1) / 2;   // 496 pairs (i, j), 1 <= j <= i < 32

// Column c by warp 0, lane i holding x = t[i][c] (updated through step c - 1): the floored
// pivot, its reciprocal square root, the scaled column, stored for the other warps and
// returned in registers for the next step.
template <class R>
__device__ __forceinline__ R tile_column(R (*t)[kT + 1], R* rs, R x, R flc, int c, bool live, int* nfloor) {
  const int lane = threadIdx.x & 31;
  R piv = r_shfl(x, c);
  if (live && !r_above(piv, flc)) {
    piv = flc;
    if (nfloor && lane == 0) atomicAdd(nfloor, 1);
  }
  const R r = r_rsqrt(piv);
  const R col = lane == c ? r_mul(piv, r) : (lane > c ? r_mul(x, r) : r_const<R>(0.0));
  if (lane >= c) t[lane][c] = col;
  if (lane == c) rs[c] = r;
  return col;
}

template <class R>
__device__ void tile_potrf(R (*t)[kT + 1], R* rs, const R* A, int64_t ld, int nn, int base, const double* diag0,
                           int* nfloor) {
  __shared__ unsigned short pairs[kTriPairs];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < kT; r += blockDim.x >> 5) {
    const int gi = base + r, gj = base + tx;
    t[r][tx] = (gi < nn && gj < nn) ? A[(int64_t)gi * ld + gj] : r_const<R>(r == tx ? 1.0 : 0.0);
  }
  // warp 0: the floor of row lane (its pivot's floor is taken by shuffle)
  const R fl = r_floor(r_const<R>(ty == 0 && base + tx < nn ? kFloorRel * fabs(diag0[base + tx]) : 0.0));
  for (int e = threadIdx.x; e < kTriPairs; e += blockDim.x) {
    int j = kT - 1, rem = e;
    while (rem >= kT - j) {
      rem -= kT - j;
      --j;
    }
    pairs[e] = (unsigned short)((j + rem) * kT + j);
  }
  __syncthreads();
  R colk = r_const<R>(0.0);
  if (ty == 0) colk = tile_column<R>(t, rs, t[tx][0], r_shfl(fl, 0), 0, base < nn, nfloor);
  __syncthreads();
  for (int k = 0; k + 1 < kT; ++k) {
    const int c = k + 1;
    if (ty == 0) {
      R x = t[tx][c];                          // column c through step k - 1
      const R lck = r_shfl(colk, c);           // L_ck
      if (tx >= c) x = r_fms(x, colk, lck);    // step k on column c
      colk = tile_column<R>(t, rs, x, r_shfl(fl, c), c, base + c < nn, nfloor);
    } else {
      const int cnt = (kT - 2 - k) * (kT - 1 - k) / 2;
      for (int e = threadIdx.x - 32; e < cnt; e += blockDim.x - 32) {
        const int i = pairs[e] / kT, j = pairs[e] % kT;
        t[i][j] = r_fms(t[i][j], t[i][k], t[j][k]);
      }
    }
    __syncthreads();
  }
}

// Panel of tile column kb: block 0 the diagonal tile, block b >= 1 rows
// [base + 32 + kPanelRows (b - 1), + kPanelRows) below it, one warp per row.  Every block loads
// the diagonal tile from A, and a block may start after block 0 has finished (when other
// kernels hold SMs), so block 0 leaves A's diagonal tile alone: its factor goes to tiles[kb]
// and the last pass (k_mirror) installs it.
template <class R>
__global__ void __launch_bounds__(kPanelThreads) k_chol_panel(R* A, int64_t ld, const int* nn_dev, int nn_fixed,
                                                              int kb, const double* diag0, int* nfloor, R* rinv,
                                                              R* tiles) {
  const int nn = dev_nn(nn_dev, nn_fixed);
  const int base = kb * kT;
  if (base >= nn) return;
  const int64_t row0 = base + kT + (int64_t)(blockIdx.x - 1) * kPanelRows;
  if (blockIdx.x > 0 && row0 >= nn) return;   // whole block: before any barrier
  __shared__ R t[kT][kT + 1];
  __shared__ R rs[kT];
  tile_potrf<R>(t, rs, A, ld, nn, base, diag0, blockIdx.x == 0 ? nfloor : nullptr);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (blockIdx.x == 0) {
    for (int r = ty; r < kT; r += kPanelThreads / 32)
      tiles[(int64_t)kb * kT * kT + r * kT + tx] = tx <= r ? t[r][tx] : r_const<R>(0.0);
    if (ty == 0 && base + tx < nn) rinv[base + tx] = rs[tx];
    return;
  }
  // row gi by warp ty: lane j holds x_j; x_c is final once scaled by 1 / L_cc
  const int64_t gi = row0 + ty;
  if (gi < nn) {
    const bool in = base + tx < nn;
    R x = in ? A[gi * ld + base + tx] : r_const<R>(0.0);
#pragma unroll 8
    for (int c = 0; c < kT; ++c) {
      if (tx == c) x = r_mul(x, rs[c]);
      const R xc = r_shfl(x, c);
      if (tx > c) x = r_fms(x, xc, t[tx][c]);
    }
    if (in) A[gi * ld + base + tx] = x;
  }
}

// 32-term dot of shared-memory rows, subtracted from a: float64 by fma; pairs accumulated
// unnormalised (high parts by two-sum, every error term into the low part), then subtracted.
__device__ __forceinline__ double dot_sub(double a, const double* x, const double* y) {
  double acc = 0.0;
#pragma unroll 8
  for (int k = 0; k < kT; ++k) acc = fma(x[k], y[k], acc);
  return a - acc;
}
__device__ __forceinline__ float2 dot_sub(float2 a, const float2* x, const float2* y) {
  float h = 0.f, l = 0.f;
#pragma unroll 8
  for (int k = 0; k < kT; ++k) df_mac(x[k], y[k], h, l);
  return df_sub_sum(a, h, l);
}

// Trailing update A_ib,jb -= L_ib,kb L_jb,kb^T for kb < jb <= ib: four blocks per tile pair,
// each a 16 x 16 quarter (one output per thread, a 32-term dot from shared memory).
template <class R>
__global__ void __launch_bounds__(256) k_chol_update(R* A, int64_t ld, const int* nn_dev, int nn_fixed, int kb) {
  const int nn = dev_nn(nn_dev, nn_fixed);
  const int nt = (nn + kT - 1) / kT;
  const int mrem = nt - kb - 1;
  const int64_t npairs = (int64_t)mrem * (mrem + 1) / 2;
  const int64_t pair = blockIdx.x >> 2;
  if (pair >= npairs) return;
  // pair -> (a, b), 0 <= b <= a < mrem, row-major over the lower triangle
  int a = (int)((sqrt(8.0 * (double)pair + 1.0) - 1.0) * 0.5);
  while ((int64_t)(a + 1) * (a + 2) / 2 <= pair) ++a;
  while ((int64_t)a * (a + 1) / 2 > pair) --a;
  const int b = (int)(pair - (int64_t)a * (a + 1) / 2);
  const int qi = (blockIdx.x >> 1) & 1, qj = blockIdx.x & 1;
  if (a == b && qj > qi) return;   // strictly upper quarter of a diagonal tile
  const int kbase = kb * kT;
  const int ibase = (kb + 1 + a) * kT + 16 * qi, jbase = (kb + 1 + b) * kT + 16 * qj;
  if (ibase >= nn || jbase >= nn) return;
  __shared__ R Li[16][kT + 1];
  __shared__ R Lj[16][kT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const bool cin = kbase + tx < nn;
  for (int r = ty; r < 16; r += 8) {
    Li[r][tx] = (ibase + r < nn && cin) ? A[(int64_t)(ibase + r) * ld + kbase + tx] : r_const<R>(0.0);
    Lj[r][tx] = (jbase + r < nn && cin) ? A[(int64_t)(jbase + r) * ld + kbase + tx] : r_const<R>(0.0);
  }
  __syncthreads();
  const int r = threadIdx.x >> 4, c = threadIdx.x & 15;
  const int gi = ibase + r, gj = jbase + c;
  if (gi < nn && gj < nn && gj <= gi) {
    R* ap = A + (int64_t)gi * ld + gj;
    *ap = dot_sub(*ap, Li[r], Lj[c]);
  }
}

// Last pass of the factorisation: the factored diagonal tiles from tiles[] (L below and on
// the diagonal, L^T above), and the upper triangle <- L^T elsewhere, so that column p of L is
// row p of the upper part.  Only diagonal tiles and the upper triangle are written; the lower
// triangle outside the diagonal tiles is only read.
template <class R>
__global__ void k_mirror(R* A, int64_t ld, const int* nn_dev, int nn_fixed, const R* tiles) {
  const int nn = nn_dev ? *nn_dev : nn_fixed;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)nn * nn; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t / nn, i = t % nn;
    if (p / kT == i / kT) {
      const R* tile = tiles + (p / kT) * kT * kT;
      const int a = (int)(p % kT), b = (int)(i % kT);
      A[p * ld + i] = b <= a ? tile[a * kT + b] : tile[b * kT + a];
    } else if (i > p) {
      A[p * ld + i] = A[i * ld + p];
    }
  }
}

// Captures the whole factorisation for an nn of at most cap (tile columns and panel rows
// beyond the device nn exit immediately).
template <class R>
static cudaError_t launch_chol(R* A, int64_t ld, const int* nn_dev, int nn_fixed, int cap, double* diag0, R* rinv,
                               R* tiles, int* nfloor, cudaStream_t st) {
  const int nt = (cap + kT - 1) / kT;
  k_chol_save_diag<R><<<std::max(1, std::min(64, (cap + 255) / 256)), 256, 0, st>>>(A, ld, nn_dev, nn_fixed, diag0,
                                                                                     nfloor);
  for (int kb = 0; kb < nt; ++kb) {
    const int rows_below = std::max(0, cap - (kb + 1) * kT);
    k_chol_panel<R><<<1 + (rows_below + kPanelRows - 1) / kPanelRows, kPanelThreads, 0, st>>>(
        A, ld, nn_dev, nn_fixed, kb, diag0, nfloor, rinv, tiles);
    const int below = nt - kb - 1;
    if (below > 0) k_chol_update<R><<<4 * below * (below + 1) / 2, 256, 0, st>>>(A, ld, nn_dev, nn_fixed, kb);
  }
  k_mirror<R><<<cap > 256 ? 256 : 64, 256, 0, st>>>(A, ld, nn_dev, nn_fixed, tiles);
  return cudaGetLastError();
}

// Inverse of every diagonal tile of the (pair) factor, L_kk^{-1} (lower, 32 x 32, row-major,
// padded by identity past nn), one block per tile: forward substitution on the identity, row c
// final once scaled by 1 / L_cc, then eliminated from the rows below.  The dense
// preconditioner's triangular solves multiply by these instead of substituting row by row.
__global__ void __launch_bounds__(256) k_chol_tile_inv(const float2* A, int64_t ld, int nn, const float2* rinv,
                                                       float2* tinv) {
  __shared__ float2 L[kT][kT + 1];
  __shared__ float2 X[kT][kT + 1];
  __shared__ float2 rs[kT];
  const int base = blockIdx.x * kT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < kT; r += 8) {
    const int gi = base + r, gj = base + tx;
    L[r][tx] = (gi < nn && gj < nn) ? (tx <= r ? A[(int64_t)gi * ld + gj] : make_float2(0.f, 0.f))
                                    : make_float2(r == tx ? 1.f : 0.f, 0.f);
    X[r][tx] = make_float2(r == tx ? 1.f : 0.f, 0.f);
  }
  if (ty == 0) rs[tx] = base + tx < nn ? rinv[base + tx] : make_float2(1.f, 0.f);
  __syncthreads();
  for (int c = 0; c < kT; ++c) {
    if (ty == 0 && tx <= c) X[c][tx] = r_mul(X[c][tx], rs[c]);
    __syncthreads();
    const int w = c + 1, cnt = (kT - 1 - c) * w;   // rows i > c, columns j <= c
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int i = c + 1 + e / w, j = e % w;
      X[i][j] = r_fms(X[i][j], L[i][c], X[c][j]);
    }
    __syncthreads();
  }
  for (int r = ty; r < kT; r += 8) tinv[(int64_t)blockIdx.x * kT * kT + r * kT + tx] = X[r][tx];
}

// Column c of A^{-1} = L^{-T} L^{-1} e_c (float64): forward sweep reads row p of the upper part
// (= column p of L), backward sweep reads row q of L; both contiguous.  One block per column at
// a time.
__global__ void k_inv(const double* A, int64_t ld, const int* nn_dev, int nn_fixed, const double* rinv, double* Ainv,
                      int64_t ldi) {
  extern __shared__ double y[];
  const int nn = nn_dev ? *nn_dev : nn_fixed;
  for (int c = blockIdx.x; c < nn; c += gridDim.x) {
    for (int i = threadIdx.x; i < nn; i += blockDim.x) y[i] = (i == c) ? 1.0 : 0.0;
    __syncthreads();
    for (int p = c; p < nn; ++p) {
      const double yp = y[p] * rinv[p];
      __syncthreads();
      if (threadIdx.x == 0) y[p] = yp;
      const double* up = A + (int64_t)p * ld;
      for (int i = p + 1 + threadIdx.x; i < nn; i += blockDim.x) y[i] = fma(-up[i], yp, y[i]);
      __syncthreads();
    }
    for (int q = nn - 1; q >= 0; --q) {
      const double xq = y[q] * rinv[q];
      __syncthreads();
      if (threadIdx.x == 0) y[q] = xq;
      const double* lq = A + (int64_t)q * ld;
      for (int i = threadIdx.x; i < q; i += blockDim.x) y[i] = fma(-lq[i], xq, y[i]);
      __syncthreads();
    }
    for (int i = threadIdx.x; i < nn; i += blockDim.x) Ainv[(int64_t)i * ldi + c] = y[i];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ forming the scaled K
// dense_aux[0] = max_ij R_ij^2 and dense_aux[1] = max |Hs| (set with the QP, as the bit
// patterns of non-negative doubles, whose unsigned order is their numeric order, so the
// atomic maximum is exact and independent of order); dense_aux[2] = the scale 2^-2e of the
// current iteration's K.

__global__ void k_dense_maxima(Dev d) {
  unsigned long long mr = 0, mh = 0;
  const int64_t nnzR = d.nR ? d.R_ptr[d.nR] : 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnzR; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = d.R_val[e] * d.R_val[e];
    mr = max(mr, (unsigned long long)__double_as_longlong(v));
  }
  const int64_t nnzH = d.Hs_ptr ? d.Hs_ptr[d.n] : 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnzH; e += (int64_t)gridDim.x * blockDim.x)
    mh = max(mh, (unsigned long long)__double_as_longlong(fabs(d.Hs_val[e])));
  unsigned long long* aux = reinterpret_cast<unsigned long long*>(d.dense_aux);
  if (mr) atomicMax(aux + 0, mr);
  if (mh) atomicMax(aux + 1, mh);
}

// One block: B = nR max_i omega_i max R^2 + max_j |h0_j + sigma_j| + max |Hs| + (a bound on
// the low-rank term) bounds every |K_ij|; s = 2^-2e with 2^2e > B puts K's entries below 1 in
// magnitude.  Then the scaled row weights as pairs, wdf_i = s omega_i.
__global__ void __launch_bounds__(1024) k_dense_prep(Dev d) {
  __shared__ double sh[32];
  __shared__ double s_scale;
  double mw = 0.0, md = 0.0, ml = 0.0;
  for (int64_t i = threadIdx.x; i < d.nR; i += blockDim.x) mw = fmax(mw, fabs(d.omega[i]));
  for (int64_t j = threadIdx.x; j < d.n; j += blockDim.x) md = fmax(md, fabs(d.h0[j] + d.sigma[j]));
  if (d.ucols)
    for (int64_t e = threadIdx.x; e < d.n * d.ucols; e += blockDim.x) {
      const double u = d.U[e];
      ml = fmax(ml, u * u * fabs(d.uw[e % d.ucols]) * (double)d.ucols);
    }
  mw = block_reduce<1>(mw, sh);
  md = block_reduce<1>(md, sh);
  ml = block_reduce<1>(ml, sh);
  if (threadIdx.x == 0) {
    const unsigned long long* aux = reinterpret_cast<const unsigned long long*>(d.dense_aux);
    const double rmax2 = __longlong_as_double((long long)aux[0]);
    const double hmax = __longlong_as_double((long long)aux[1]);
    const double B = mw * rmax2 * (double)(d.nR > 0 ? d.nR : 1) + md + hmax + ml;
    int e = 0;
    if (B > 0.0 && isfinite(B)) {
      frexp(B, &e);   // B < 2^e
      e += e & 1;     // even: the factor's scale 2^-e/2 is exact too
    }
    s_scale = ldexp(1.0, -e);
    d.dense_aux[2] = s_scale;
  }
  __syncthreads();
  const double s = s_scale;
  for (int64_t i = threadIdx.x; i < d.nR; i += blockDim.x) d.wdf[i] = df_split(s * d.omega[i]);
}

// K = R^T diag(omega) R + U W U^T (scaled, as pairs) by 32 x 32 tiles: one block per tile of
// the lower triangle, 2 x 2 outputs per thread, each a sum in row order, so K is
// deterministic; off-diagonal tiles are written to both triangles.
constexpr int kGT = 32;

__device__ __forceinline__ void tile_of_block(int64_t b, int64_t& tj, int64_t& tl) {
  tj = (int64_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while ((tj + 1) * (tj + 2) / 2 <= b) ++tj;
  while (tj * (tj + 1) / 2 > b) --tj;
  tl = b - tj * (tj + 1) / 2;
}

// the low-rank term's columns into the 2 x 2 accumulators (sJ, sL: 32 pairs of shared
// memory each)
__device__ __forceinline__ void gram_lowrank_acc(const Dev& d, int64_t J0, int64_t L0, float2* sJ, float2* sL,
                                                 float (&h)[2][2], float (&l)[2][2]) {
  const int64_t n = d.n;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const double s = d.dense_aux[2];
  for (int64_t r = 0; r < d.ucols; ++r) {
    __syncthreads();
    if (tid < kGT) {
      sJ[tid] = J0 + tid < n ? df_split(d.U[(J0 + tid) * d.ucols + r] * d.uw[r] * s) : make_float2(0.f, 0.f);
      sL[tid] = L0 + tid < n ? df_split(d.U[(L0 + tid) * d.ucols + r]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = 0; c < 2; ++c) df_mac(sJ[2 * ty + a], sL[2 * tx + c], h[a][c], l[a][c]);
  }
}

// the tile's stores (both triangles off the diagonal)
__device__ __forceinline__ void gram_store(const Dev& d, int64_t J0, int64_t L0, int64_t tj, int64_t tl,
                                           const float (&h)[2][2], const float (&l)[2][2]) {
  const int64_t n = d.n;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int64_t j = J0 + 2 * ty + a, lc = L0 + 2 * tx + c;
      if (j < n && lc < n) {
        const float2 v = df_fast_sum(h[a][c], l[a][c]);
        d.Kd[j * n + lc] = v;
        if (tj != tl) d.Kd[lc * n + j] = v;
      }
    }
}

// From the CSR rows of R (when R is too large to keep densely): for every row i the block
// gathers the row's entries that fall in its two column ranges (one side scaled by the row
// weight) and adds their outer product.
__global__ void __launch_bounds__(256) k_gram_tiles(Dev d) {
  __shared__ float2 sJ[kGT], sL[kGT];
  int64_t tj, tl;
  tile_of_block(blockIdx.x, tj, tl);
  const int64_t J0 = tj * kGT, L0 = tl * kGT;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float h[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, l[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int64_t i = 0; i < d.nR; ++i) {
    if (tid < kGT) {
      sJ[tid] = make_float2(0.f, 0.f);
      sL[tid] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2 w = d.wdf[i];
    int hj = 0, hl = 0;
    if (w.x != 0.f) {
      for (int64_t e = d.R_ptr[i] + tid; e < d.R_ptr[i + 1]; e += blockDim.x) {
        const int64_t c = d.R_idx[e];
        if (c >= J0 && c < J0 + kGT) {
          sJ[c - J0] = r_mul(w, df_split(d.R_val[e]));
          hj = 1;
        }
        if (c >= L0 && c < L0 + kGT) {
          sL[c - L0] = df_split(d.R_val[e]);
          hl = 1;
        }
      }
    }
    hj = __syncthreads_or(hj);
    hl = __syncthreads_or(hl);
    if (hj && hl) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c) df_mac(sJ[2 * ty + a], sL[2 * tx + c], h[a][c], l[a][c]);
    }
    __syncthreads();
  }
  gram_lowrank_acc(d, J0, L0, sJ, sL, h, l);
  gram_store(d, J0, L0, tj, tl, h, l);
}

// From the dense copy of R (pairs): chunks of 32 rows of Rd staged in shared memory (one side
// scaled by the row weight), rows summed in order.  The next chunk is loaded into registers
// while the current one is multiplied.
// With row splits (gridDim.y > 1) block (t, s) sums the rows of chunk range s of tile t and
// writes its unnormalised pairs to gram_part[s][t] (split 0 also takes the low-rank term);
// k_gram_sum adds the splits in order.
__global__ void __launch_bounds__(256) k_gram_gemm(Dev d) {
  __shared__ float2 sA[kGT][kGT + 1], sB[kGT][kGT + 1];
  const int64_t n = d.n;
  int64_t tj, tl;
  tile_of_block(blockIdx.x, tj, tl);
  const int64_t chunks = (d.nR + kGT - 1) / kGT, per = (chunks + gridDim.y - 1) / gridDim.y;
  const int64_t r_beg = blockIdx.y * per * kGT, r_end = min(d.nR, (int64_t)(blockIdx.y + 1) * per * kGT);
  const int64_t J0 = tj * kGT, L0 = tl * kGT;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float h[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, l[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  constexpr int kPer = kGT * kGT / 256;   // staged entries per thread and side
  float2 ra[kPer], rb[kPer];
  auto fetch = [&](int64_t i0) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int t = tid + q * 256, ii = t >> 5, cc = t & 31;
      const int64_t i = i0 + ii;
      const bool in = i < r_end;
      ra[q] = (in && J0 + cc < n) ? r_mul(d.Rd[i * n + J0 + cc], d.wdf[i]) : make_float2(0.f, 0.f);
      rb[q] = (in && L0 + cc < n) ? d.Rd[i * n + L0 + cc] : make_float2(0.f, 0.f);
    }
  };
  if (r_beg < r_end) fetch(r_beg);
  for (int64_t i0 = r_beg; i0 < r_end; i0 += kGT) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int t = tid + q * 256;
      sA[t >> 5][t & 31] = ra[q];
      sB[t >> 5][t & 31] = rb[q];
    }
    __syncthreads();
    if (i0 + kGT < r_end) fetch(i0 + kGT);
#pragma unroll 4
    for (int ii = 0; ii < kGT; ++ii) {
      const float2 a0 = sA[ii][2 * ty], a1 = sA[ii][2 * ty + 1];
      const float2 b0 = sB[ii][2 * tx], b1 = sB[ii][2 * tx + 1];
      df_mac(a0, b0, h[0][0], l[0][0]);
      df_mac(a0, b1, h[0][1], l[0][1]);
      df_mac(a1, b0, h[1][0], l[1][0]);
      df_mac(a1, b1, h[1][1], l[1][1]);
    }
    __syncthreads();
  }
  if (blockIdx.y == 0) gram_lowrank_acc(d, J0, L0, &sA[0][0], &sB[0][0], h, l);
  if (gridDim.y == 1) {
    gram_store(d, J0, L0, tj, tl, h, l);
    return;
  }
  float2* part = d.gram_part + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * kGT * kGT;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) part[(2 * ty + a) * kGT + 2 * tx + c] = make_float2(h[a][c], l[a][c]);
}

// The row splits' partial tiles added in split order (two-sum of the high parts, the low parts
// and errors summed), one thread per tile entry; the tile stores as k_gram_gemm's.
__global__ void k_gram_sum(Dev d, int splits, int64_t tiles) {
  const int64_t n = d.n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tiles * kGT * kGT;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tile = t / (kGT * kGT);
    const int e = (int)(t % (kGT * kGT)), a = e / kGT, c = e % kGT;
    int64_t tj, tl;
    tile_of_block(tile, tj, tl);
    const int64_t j = tj * kGT + a, lc = tl * kGT + c;
    if (j >= n || lc >= n) continue;
    float h = 0.f, l = 0.f;
    for (int s = 0; s < splits; ++s) {
      const float2 p = d.gram_part[((int64_t)s * tiles + tile) * kGT * kGT + e];
      float sum, err;
      two_sum(h, p.x, sum, err);
      h = sum;
      l = __fadd_rn(l, __fadd_rn(err, p.y));
    }
    const float2 v = df_fast_sum(h, l);
    d.Kd[j * n + lc] = v;
    if (tj != tl) d.Kd[lc * n + j] = v;
  }
}

__global__ void k_densify_zero(float2* Rd, int64_t total) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    Rd[t] = make_float2(0.f, 0.f);
}

__global__ void k_densify_fill(Dev d) {
  for (int64_t r = blockIdx.x; r < d.nR; r += gridDim.x)
    for (int64_t e = d.R_ptr[r] + threadIdx.x; e < d.R_ptr[r + 1]; e += blockDim.x)
      d.Rd[r * d.n + d.R_idx[e]] = df_split(d.R_val[e]);
}

cudaError_t launch_densify_R(const Dev& d, cudaStream_t st) {
  if (!d.Kd) return cudaSuccess;
  cudaMemsetAsync(d.dense_aux, 0, 4 * sizeof(double), st);
  k_dense_maxima<<<4 * 152, 256, 0, st>>>(d);
  if (!d.Rd || !d.nR) return cudaGetLastError();
  k_densify_zero<<<1024, 256, 0, st>>>(d.Rd, d.nR * d.n);
  k_densify_fill<<<(int)std::min<int64_t>(d.nR, 4096), 256, 0, st>>>(d);
  return cudaGetLastError();
}

// Adds s (diag(h0 + sigma) + Hs) (each entry once: no conflicts), in float64 on the pair.
__global__ void k_gram_diag_hs(Dev d) {
  const int64_t n = d.n;
  const double s = d.dense_aux[2];
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    if (threadIdx.x == 0) {
      float2* kp = d.Kd + j * n + j;
      *kp = df_split(df_value(kp->x, kp->y) + s * (d.h0[j] + d.sigma[j]));
    }
    if (d.Hs_ptr) {
      __syncthreads();
      for (int64_t e = d.Hs_ptr[j] + threadIdx.x; e < d.Hs_ptr[j + 1]; e += blockDim.x) {
        float2* kp = d.Kd + j * n + d.Hs_idx[e];
        *kp = df_split(df_value(kp->x, kp->y) + s * d.Hs_val[e]);
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_dense_build(const Dev& d, cudaStream_t st) {
  const int n = (int)d.n;
  const int64_t nt = (d.n + kGT - 1) / kGT;
  k_dense_prep<<<1, 1024, 0, st>>>(d);
  if (d.Rd) {
    const int splits = d.gram_part ? gram_splits(d.n) : 1;
    const int64_t tiles = nt * (nt + 1) / 2;
    k_gram_gemm<<<dim3((unsigned)tiles, (unsigned)splits), 256, 0, st>>>(d);
    if (splits > 1) k_gram_sum<<<(unsigned)std::min<int64_t>((tiles * 1024 + 255) / 256, 4 * 152), 256, 0, st>>>(d, splits, tiles);
  } else
    k_gram_tiles<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, st>>>(d);
  k_gram_diag_hs<<<(int)std::min<int64_t>(d.n, 4 * 152), 256, 0, st>>>(d);
  cudaError_t e = launch_chol<float2>(d.Kd, d.n, nullptr, n, n, d.chol_diag, d.chol_rdf,
                                      reinterpret_cast<float2*>(d.chol_tiles), &d.sc->chol_fail, st);
  if (e != cudaSuccess) return e;
  if (nt > 0) k_chol_tile_inv<<<(unsigned)nt, 256, 0, st>>>(d.Kd, d.n, n, d.chol_rdf, d.chol_tinv);
  return cudaGetLastError();
}

cudaError_t launch_stiff_factor(const Dev& d, cudaStream_t st) {
  const int cap = d.stiff_cap;
  const size_t rowbytes = sizeof(double) * (size_t)cap;
  const int* ns = &d.sc->n_stiff;
  cudaError_t e = launch_chol<double>(d.G, cap, ns, 0, cap, d.chol_diag, d.chol_rinv, d.chol_tiles,
                                      &d.sc->chol_fail, st);
  if (e != cudaSuccess) return e;
  k_inv<<<std::min(cap, 4 * 152), 256, rowbytes, st>>>(d.G, cap, ns, 0, d.chol_rinv, d.Ginv, cap);
  return cudaGetLastError();
}

}  // namespace ipmk
