// Dense pieces of the preconditioners (sm_103a, float64):
//   * k_gram_tiles / k_gram_diag_hs : K = Hs + R^T diag(omega) R + U W U^T + diag(h0 + sigma) as a
//                  dense n x n matrix
//                  (the DENSE preconditioner: one diagonal block covering all variables);
//   * k_chol_*   : in-place blocked Cholesky factor (lower) with pivot flooring, and the
//                  reciprocal pivots;
//   * k_mirror   : copies L into the upper triangle so both triangular sweeps read rows;
//   * k_inv      : explicit inverse from the factor, columns spread over blocks.
// The low-rank correction's G (up to 1024 rows) is inverted explicitly, so each of the many
// PCG applies is a parallel matvec; the DENSE preconditioner, whose PCG takes one or two
// iterations, is applied by triangular solves with the factor instead.  The factorisation
// runs once per IPM iteration.
#include <algorithm>
#include <cmath>

#include "state.h"

namespace ipmk {


// Blocked right-looking Cholesky (lower, row-major, leading dimension ld) of the leading
// nn x nn block of A on 32 x 32 tiles, two launches per tile column kb:
//   * the panel: every block factors the diagonal tile in shared memory (the same code on the
//     same data, so each gets the same factor; block 0 writes it back), then the others each
//     solve 8 rows of the tiles below, X = A_ib,kb L_kb,kb^{-T}, one warp per row;
//   * the trailing update A_ib,jb -= L_ib,kb L_jb,kb^T (kb < jb <= ib) on 16 x 16 quarter tiles.
// GB300's float64 pipe issues two fused multiply-adds per SM per clock, so a 32-step chain
// of float64 operations on one warp costs tens of microseconds: each pivot takes one rsqrt
// and the rest multiplies by it (no division on the chain), and the arithmetic of a tile
// column is spread over as many SMs as it has row blocks.  The reciprocal pivots go to
// rinv[] for the triangular solves.  nn is read on the device (it may be the number of stiff
// rows).  A pivot below floor_rel * (original diagonal) is raised to that floor (a modified
// factor; still symmetric positive definite, which is all a preconditioner needs); the count
// goes to *nfloor.
constexpr int kT = 32;
constexpr int kPanelRows = 8;   // rows of the panel below the diagonal tile per block

__device__ __forceinline__ int dev_nn(const int* nn_dev, int nn_fixed) { return nn_dev ? *nn_dev : nn_fixed; }

__global__ void k_chol_save_diag(const double* A, int64_t ld, const int* nn_dev, int nn_fixed, double* diag0, int* nfloor) {
  const int nn = dev_nn(nn_dev, nn_fixed);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) diag0[i] = A[(int64_t)i * ld + i];
  if (blockIdx.x == 0 && threadIdx.x == 0 && nfloor) *nfloor = 0;
}

// Unblocked Cholesky of diagonal tile kb in shared memory by 256 threads (rows/cols >= nn
// padded by identity): rs[k] = 1 / L_kk.  Pivots are floored as above; nfloor (may be null)
// counts the floored ones.
__device__ void tile_potrf(double (*t)[kT + 1], double* rs, const double* A, int64_t ld, int nn, int base,
                           const double* diag0, double floor_rel, int* nfloor) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  for (int r = ty; r < kT; r += 8) {
    const int gi = base + r, gj = base + tx;
    t[r][tx] = (gi < nn && gj < nn) ? A[(int64_t)gi * ld + gj] : (r == tx ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int k = 0; k < kT; ++k) {
    if (ty == 0) {   // column k by warp 0
      double piv = t[k][k];
      __syncwarp();
      if (base + k < nn) {
        const double fl = floor_rel * fabs(diag0[base + k]) + 1e-300;
        if (!(piv > fl)) {
          piv = fl;
          if (nfloor && tx == 0) atomicAdd(nfloor, 1);
        }
      }
      const double r = rsqrt(piv);
      if (tx == k) {
        t[k][k] = piv * r;
        rs[k] = r;
      } else if (tx > k) {
        t[tx][k] *= r;
      }
    }
    __syncthreads();
    for (int i = k + 1 + ty; i < kT; i += 8)
      if (tx > k && tx <= i) t[i][tx] = fma(-t[i][k], t[tx][k], t[i][tx]);
    __syncthreads();
  }
}

// Panel of tile column kb: block 0 the diagonal tile, block b >= 1 rows
// [base + 32 + 8 (b - 1), + 8) below it.
__global__ void __launch_bounds__(256) k_chol_panel(double* A, int64_t ld, const int* nn_dev, int nn_fixed, int kb,
                                                    const double* diag0, double floor_rel, int* nfloor, double* rinv) {
  const int nn = dev_nn(nn_dev, nn_fixed);
  const int base = kb * kT;
  if (base >= nn) return;
  const int64_t row0 = base + kT + (int64_t)(blockIdx.x - 1) * kPanelRows;
  if (blockIdx.x > 0 && row0 >= nn) return;   // whole block: before any barrier
  __shared__ double t[kT][kT + 1];
  __shared__ double rs[kT];
  tile_potrf(t, rs, A, ld, nn, base, diag0, floor_rel, blockIdx.x == 0 ? nfloor : nullptr);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (blockIdx.x == 0) {
    for (int r = ty; r < kT; r += 8) {
      const int gi = base + r, gj = base + tx;
      if (gi < nn && gj < nn && tx <= r) A[(int64_t)gi * ld + gj] = t[r][tx];
    }
    if (ty == 0 && base + tx < nn) rinv[base + tx] = rs[tx];
    return;
  }
  // row gi by warp ty: lane j holds x_j; x_c is final once scaled by 1 / L_cc
  const int64_t gi = row0 + ty;
  if (gi < nn) {
    const bool in = base + tx < nn;
    double x = in ? A[gi * ld + base + tx] : 0.0;
#pragma unroll 8
    for (int c = 0; c < kT; ++c) {
      if (tx == c) x *= rs[c];
      const double xc = __shfl_sync(0xffffffffu, x, c);
      if (tx > c) x = fma(-xc, t[tx][c], x);
    }
    if (in) A[gi * ld + base + tx] = x;
  }
}

// Trailing update A_ib,jb -= L_ib,kb L_jb,kb^T for kb < jb <= ib: four blocks per tile pair,
// each a 16 x 16 quarter (one output per thread, a 32-term dot from shared memory).
__global__ void __launch_bounds__(256) k_chol_update(double* A, int64_t ld, const int* nn_dev, int nn_fixed, int kb) {
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
  __shared__ double Li[16][kT + 1];
  __shared__ double Lj[16][kT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const bool cin = kbase + tx < nn;
  for (int r = ty; r < 16; r += 8) {
    Li[r][tx] = (ibase + r < nn && cin) ? A[(int64_t)(ibase + r) * ld + kbase + tx] : 0.0;
    Lj[r][tx] = (jbase + r < nn && cin) ? A[(int64_t)(jbase + r) * ld + kbase + tx] : 0.0;
  }
  __syncthreads();
  const int r = threadIdx.x >> 4, c = threadIdx.x & 15;
  const int gi = ibase + r, gj = jbase + c;
  if (gi < nn && gj < nn && gj <= gi) {
    double acc = 0.0;
#pragma unroll 8
    for (int k = 0; k < kT; ++k) acc = fma(Li[r][k], Lj[c][k], acc);
    A[(int64_t)gi * ld + gj] -= acc;
  }
}

// Captures the whole factorisation for an nn of at most cap (tile columns and panel rows
// beyond the device nn exit immediately).
static cudaError_t launch_chol(double* A, int64_t ld, const int* nn_dev, int nn_fixed, int cap, double* diag0,
                               double* rinv, int* nfloor, cudaStream_t st) {
  const int nt = (cap + kT - 1) / kT;
  k_chol_save_diag<<<std::max(1, std::min(64, (cap + 255) / 256)), 256, 0, st>>>(A, ld, nn_dev, nn_fixed, diag0, nfloor);
  for (int kb = 0; kb < nt; ++kb) {
    const int rows_below = std::max(0, cap - (kb + 1) * kT);
    k_chol_panel<<<1 + (rows_below + kPanelRows - 1) / kPanelRows, 256, 0, st>>>(A, ld, nn_dev, nn_fixed, kb, diag0,
                                                                                   1e-13, nfloor, rinv);
    const int below = nt - kb - 1;
    if (below > 0) k_chol_update<<<4 * below * (below + 1) / 2, 256, 0, st>>>(A, ld, nn_dev, nn_fixed, kb);
  }
  return cudaGetLastError();
}

// Upper triangle <- L^T so that column p of L is row p of the upper part.
__global__ void k_mirror(double* A, int64_t ld, const int* nn_dev, int nn_fixed) {
  const int nn = nn_dev ? *nn_dev : nn_fixed;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)nn * nn; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t / nn, i = t % nn;
    if (i > p) A[p * ld + i] = A[i * ld + p];
  }
}

// Column c of A^{-1} = L^{-T} L^{-1} e_c: forward sweep reads row p of the upper part (= column
// p of L), backward sweep reads row q of L; both contiguous.  One block per column at a time.
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

// K = R^T diag(omega) R + U W U^T + Hs + diag(h0 + sigma) by 32 x 32 tiles: one block per
// tile of the lower triangle; for every row i of R (in order) the block gathers the row's
// entries that fall in its two column ranges (scaled by omega_i on one side) and adds their
// outer product (2 x 2 outputs per thread); the columns of U likewise.  Each output is a sum
// in row order, so K is deterministic; off-diagonal tiles are written to both triangles.
constexpr int kGT = 32;

__global__ void __launch_bounds__(256) k_gram_tiles(Dev d) {
  __shared__ double sJ[kGT], sL[kGT];
  const int64_t n = d.n;
  const int64_t b = blockIdx.x;
  int64_t tj = (int64_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while ((tj + 1) * (tj + 2) / 2 <= b) ++tj;
  while (tj * (tj + 1) / 2 > b) --tj;
  const int64_t tl = b - tj * (tj + 1) / 2;
  const int64_t J0 = tj * kGT, L0 = tl * kGT;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t i = 0; i < d.nR; ++i) {
    if (tid < kGT) { sJ[tid] = 0.0; sL[tid] = 0.0; }
    __syncthreads();
    const double w = d.omega[i];
    int hj = 0, hl = 0;
    if (w != 0.0) {
      for (int64_t e = d.R_ptr[i] + tid; e < d.R_ptr[i + 1]; e += blockDim.x) {
        const int64_t c = d.R_idx[e];
        const double v = d.R_val[e];
        if (c >= J0 && c < J0 + kGT) { sJ[c - J0] = w * v; hj = 1; }
        if (c >= L0 && c < L0 + kGT) { sL[c - L0] = v; hl = 1; }
      }
    }
    hj = __syncthreads_or(hj);
    hl = __syncthreads_or(hl);
    if (hj && hl) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c) acc[a][c] = fma(sJ[2 * ty + a], sL[2 * tx + c], acc[a][c]);
    }
    __syncthreads();
  }
  for (int64_t r = 0; r < d.ucols; ++r) {
    if (tid < kGT) {
      sJ[tid] = J0 + tid < n ? d.U[(J0 + tid) * d.ucols + r] * d.uw[r] : 0.0;
      sL[tid] = L0 + tid < n ? d.U[(L0 + tid) * d.ucols + r] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = 0; c < 2; ++c) acc[a][c] = fma(sJ[2 * ty + a], sL[2 * tx + c], acc[a][c]);
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int64_t j = J0 + 2 * ty + a, l = L0 + 2 * tx + c;
      if (j < n && l < n) {
        d.Kd[j * n + l] = acc[a][c];
        if (tj != tl) d.Kd[l * n + j] = acc[a][c];
      }
    }
}

// The same tiles from the dense copy of R: chunks of 32 rows of Rd staged in shared memory
// (one side scaled by omega), 2 x 2 outputs per thread, rows summed in order; plus U W U^T.
__global__ void __launch_bounds__(256) k_gram_gemm(Dev d) {
  __shared__ double sA[kGT][kGT + 1], sB[kGT][kGT + 1];
  const int64_t n = d.n;
  const int64_t b = blockIdx.x;
  int64_t tj = (int64_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while ((tj + 1) * (tj + 2) / 2 <= b) ++tj;
  while (tj * (tj + 1) / 2 > b) --tj;
  const int64_t tl = b - tj * (tj + 1) / 2;
  const int64_t J0 = tj * kGT, L0 = tl * kGT;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t i0 = 0; i0 < d.nR; i0 += kGT) {
    for (int t = tid; t < kGT * kGT; t += blockDim.x) {
      const int ii = t >> 5, cc = t & 31;
      const int64_t i = i0 + ii;
      const bool in = i < d.nR;
      sA[ii][cc] = (in && J0 + cc < n) ? d.Rd[i * n + J0 + cc] * d.omega[i] : 0.0;
      sB[ii][cc] = (in && L0 + cc < n) ? d.Rd[i * n + L0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int ii = 0; ii < kGT; ++ii) {
      const double a0 = sA[ii][2 * ty], a1 = sA[ii][2 * ty + 1];
      const double b0 = sB[ii][2 * tx], b1 = sB[ii][2 * tx + 1];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  for (int64_t r = 0; r < d.ucols; ++r) {
    if (tid < kGT) {
      sA[0][tid] = J0 + tid < n ? d.U[(J0 + tid) * d.ucols + r] * d.uw[r] : 0.0;
      sB[0][tid] = L0 + tid < n ? d.U[(L0 + tid) * d.ucols + r] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = 0; c < 2; ++c) acc[a][c] = fma(sA[0][2 * ty + a], sB[0][2 * tx + c], acc[a][c]);
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int64_t j = J0 + 2 * ty + a, l = L0 + 2 * tx + c;
      if (j < n && l < n) {
        d.Kd[j * n + l] = acc[a][c];
        if (tj != tl) d.Kd[l * n + j] = acc[a][c];
      }
    }
}

__global__ void k_densify_zero(double* Rd, int64_t total) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    Rd[t] = 0.0;
}

__global__ void k_densify_fill(Dev d) {
  for (int64_t r = blockIdx.x; r < d.nR; r += gridDim.x)
    for (int64_t e = d.R_ptr[r] + threadIdx.x; e < d.R_ptr[r + 1]; e += blockDim.x) d.Rd[r * d.n + d.R_idx[e]] = d.R_val[e];
}

cudaError_t launch_densify_R(const Dev& d, cudaStream_t st) {
  if (!d.Rd || !d.nR) return cudaSuccess;
  k_densify_zero<<<1024, 256, 0, st>>>(d.Rd, d.nR * d.n);
  k_densify_fill<<<(int)std::min<int64_t>(d.nR, 4096), 256, 0, st>>>(d);
  return cudaGetLastError();
}

// Adds diag(h0 + sigma) and the explicit block Hs (each entry once: no conflicts).
__global__ void k_gram_diag_hs(Dev d) {
  const int64_t n = d.n;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    if (threadIdx.x == 0) d.Kd[j * n + j] += d.h0[j] + d.sigma[j];
    if (d.Hs_ptr) {
      __syncthreads();
      for (int64_t e = d.Hs_ptr[j] + threadIdx.x; e < d.Hs_ptr[j + 1]; e += blockDim.x) d.Kd[j * n + d.Hs_idx[e]] += d.Hs_val[e];
    }
    __syncthreads();
  }
}

cudaError_t launch_dense_build(const Dev& d, cudaStream_t st) {
  const int n = (int)d.n;
  const size_t rowbytes = sizeof(double) * (size_t)n;
  const int64_t nt = (d.n + kGT - 1) / kGT;
  if (d.Rd)
    k_gram_gemm<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, st>>>(d);
  else
    k_gram_tiles<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, st>>>(d);
  k_gram_diag_hs<<<(int)std::min<int64_t>(d.n, 4 * 152), 256, 0, st>>>(d);
  cudaError_t e = launch_chol(d.Kd, d.n, nullptr, n, n, d.chol_diag, d.chol_rinv, &d.sc->chol_fail, st);
  if (e != cudaSuccess) return e;
  k_mirror<<<256, 256, 0, st>>>(d.Kd, d.n, nullptr, n);
  (void)rowbytes;   // applied by triangular solves (k_dense_trsv), no explicit inverse
  return cudaGetLastError();
}

cudaError_t launch_stiff_factor(const Dev& d, cudaStream_t st) {
  const int cap = d.stiff_cap;
  const size_t rowbytes = sizeof(double) * (size_t)cap;
  const int* ns = &d.sc->n_stiff;
  cudaError_t e = launch_chol(d.G, cap, ns, 0, cap, d.chol_diag, d.chol_rinv, &d.sc->chol_fail, st);
  if (e != cudaSuccess) return e;
  k_mirror<<<64, 256, 0, st>>>(d.G, cap, ns, 0);
  k_inv<<<std::min(cap, 4 * 152), 256, rowbytes, st>>>(d.G, cap, ns, 0, d.chol_rinv, d.Ginv, cap);
  return cudaGetLastError();
}

}  // namespace ipmk
