// sm_103a kernels of the interior point method: residuals, diagonal update, right-hand side,
// the matrix-free PCG iteration, direction recovery, ratio test and update.
//
// Operator (the condensed form of the paper's KKT matvec, Section 4.1.1 / Listing 1):
//     K p = R^T (omega o (R p)) + Hs p + (h0 + sigma) o p,
// where R = [F; A_csr] and omega = w_R + theta placed on the constraint rows, so that
// R^T diag(omega) R = F^T W F + A^T Theta A.  One PCG iteration is two streaming passes:
// k_op_rows (row gather over R) and k_op_cols (row gather over the stored transpose R^T).
// All reductions are block-tree + last-block sums in block order: results are bitwise
// reproducible for a fixed problem size.
#include <algorithm>
#include <cmath>

#include "state.h"

namespace ipmk {

static __device__ __forceinline__ int gwarp() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
static __device__ __forceinline__ int nwarps() { return (gridDim.x * blockDim.x) >> 5; }

// Lanes per row of the streaming row kernels (see group_row_dot): G is a template parameter,
// picked per matrix at ipm_set_qp (Dev::g_rows for R, Dev::g_cols for R^T).
template <int G>
static __device__ __forceinline__ int glane() { return threadIdx.x & (G - 1); }

// Grid-stride loop over rows, G lanes per row, with a warp-uniform trip count (the group
// shuffles need every lane of the warp): the loop runs over the first row of each warp's
// groups; a group whose row is past the end works on an empty row.
#define FOR_GROUP_ROWS(G, r, ok, nrows)                                                                \
  for (int64_t r##_0 = (int64_t)gwarp() * (32 / G); r##_0 < (nrows); r##_0 += (int64_t)nwarps() * (32 / G)) \
    for (int64_t r = r##_0 + (threadIdx.x & 31) / G, r##_once = 0; r##_once == 0; r##_once = 1)           \
      for (bool ok = r < (nrows), ok##_once = true; ok##_once; ok##_once = false)

// Instantiates a launch for the lane-group size g (4, 8, 16 or 32) chosen at run time.
#define DISPATCH_G(g, ...)                         \
  do {                                             \
    switch (g) {                                   \
      case 4: { constexpr int G = 4; __VA_ARGS__; } break;   \
      case 8: { constexpr int G = 8; __VA_ARGS__; } break;   \
      case 16: { constexpr int G = 16; __VA_ARGS__; } break; \
      default: { constexpr int G = 32; __VA_ARGS__; } break; \
    }                                              \
  } while (0)


Geo make_geo(const Dev& d) {
  // at most 8 blocks of 256 threads per SM (the row kernels are grid-stride loops)
  const int cap = std::min(kMaxRedBlocks, 8 * (d.sm_count > 0 ? d.sm_count : 148));
  auto blocks_for = [cap](int64_t items, int per_block) -> int {
    int64_t b = (items + per_block - 1) / per_block;
    if (b > cap) b = cap;
    return (int)b;
  };
  Geo g;
  const int gr = d.g_rows > 0 ? d.g_rows : 32, gc = d.g_cols > 0 ? d.g_cols : 32;
  g.gR = blocks_for(d.nR, kBlock / gr);
  g.gM = blocks_for(d.m, kBlock / gr);
  g.gN = blocks_for(d.n, kBlock / gc);
  g.eM = blocks_for(d.m, kBlock);
  g.eN = blocks_for(d.n, kBlock);
  // the PCG column kernels are limited to 40 registers (6 blocks per SM): one full wave
  g.gNc = (int)std::min<int64_t>(g.gN, 6 * (int64_t)(d.sm_count > 0 ? d.sm_count : 148));
  g.gRc = (int)std::min<int64_t>(g.gR, 6 * (int64_t)(d.sm_count > 0 ? d.sm_count : 148));
  g.gR64 = (int)std::min<int64_t>(g.gR, kOpRowsMinBlocks * (int64_t)(d.sm_count > 0 ? d.sm_count : 148));
  g.gN64 = (int)std::min<int64_t>(g.gN, kOpColsMinBlocks * (int64_t)(d.sm_count > 0 ? d.sm_count : 148));
  // the residual and right-hand-side column kernels are limited to 64 registers (4 per SM)
  g.gNr = (int)std::min<int64_t>(g.gN, 4 * (int64_t)(d.sm_count > 0 ? d.sm_count : 148));
  return g;
}

// ------------------------------------------------------------------------------ low-rank term

// H's low-rank term U W U^T (eq:bfgs_hessian: H = H0 + U W U^T, U dense n x 2k, W diagonal) is
// applied matrix-free in two dense passes over U: t = U^T v (this pair of kernels, a
// reduction over the n rows of U split into row chunks, one partial vector per block, summed
// in block order), then (U (W t))_j inside the column kernels (lr_row).  Row-major U makes
// both passes read rows of U contiguously.
__global__ void __launch_bounds__(256) k_lr_part(Dev d, const double* __restrict__ v) {
  // 8 warps per block; warp w takes rows j0 + w, j0 + w + 8, ... of the block's chunk; lane l
  // accumulates columns r0 + l + 32 c (c < 4) of a 128-column slice; the warps' sums are
  // added in warp order through shared memory.
  constexpr int RC = 4;
  __shared__ double sh[8][32 * RC];
  const int64_t uc = d.ucols, n = d.n;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t j0 = (int64_t)blockIdx.x * per, j1 = j0 + per < n ? j0 + per : n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t r0 = 0; r0 < uc; r0 += 32 * RC) {
    double acc[RC];
#pragma unroll
    for (int c = 0; c < RC; ++c) acc[c] = 0.0;
    int64_t j = j0 + w;
    for (; j + 8 < j1; j += 16) {
      const double* u0 = d.U + j * uc + r0 + lane;
      const double* u1 = u0 + 8 * uc;
      const double x0 = __ldg(v + j), x1 = __ldg(v + j + 8);
      double t0[RC], t1[RC];
#pragma unroll
      for (int c = 0; c < RC; ++c) {
        const bool in = r0 + lane + 32 * c < uc;
        t0[c] = in ? __ldg(u0 + 32 * c) : 0.0;
        t1[c] = in ? __ldg(u1 + 32 * c) : 0.0;
      }
#pragma unroll
      for (int c = 0; c < RC; ++c) acc[c] = fma(t1[c], x1, fma(t0[c], x0, acc[c]));
    }
    if (j < j1) {
      const double* u0 = d.U + j * uc + r0 + lane;
      const double x0 = __ldg(v + j);
#pragma unroll
      for (int c = 0; c < RC; ++c)
        if (r0 + lane + 32 * c < uc) acc[c] = fma(__ldg(u0 + 32 * c), x0, acc[c]);
    }
#pragma unroll
    for (int c = 0; c < RC; ++c) sh[w][lane + 32 * c] = acc[c];
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * RC; t += blockDim.x) {
      if (r0 + t < uc) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) s += sh[q][t];
        d.upart[(r0 + t) * (int64_t)d.ublocks + blockIdx.x] = s;   // column-major: the final sum reads runs
      }
    }
    __syncthreads();
  }
}

// lrs = uw o t, t_r = the sum of the block partials of column r (stored column-major; one warp
// per r: lane l adds the partials of blocks l, l + 32, ..., then a fixed shuffle tree);
// quad: lrq_r = uw_r t_r^2.
__global__ void k_lr_final(Dev d, int quad) {
  const int64_t uc = d.ucols;
  const int lane = threadIdx.x & 31;
  for (int64_t r = gwarp(); r < uc; r += nwarps()) {
    double t = 0.0;
    for (int b = lane; b < d.ublocks; b += 32) t += d.upart[r * (int64_t)d.ublocks + b];
    t = warp_sum(t);
    if (lane == 0) {
      const double sv = d.uw[r] * t;
      d.lrs[r] = sv;
      if (quad) d.lrq[r] = sv * t;
    }
  }
}

// v^T U W U^T v = sum_r lrq_r (one block, fixed order) into the device scalars.
__global__ void k_lr_quad(Dev d) {
  __shared__ double sh[32];
  double q = 0.0;
  for (int64_t r = threadIdx.x; r < d.ucols; r += blockDim.x) q += d.lrq[r];
  q = block_reduce<0>(q, sh);
  if (threadIdx.x == 0) d.sc->lr_quad = q;
}

cudaError_t launch_lr(const Dev& d, const double* v, int quad, cudaStream_t st) {
  if (!d.ucols) return cudaSuccess;
  k_lr_part<<<d.ublocks, 256, 0, st>>>(d, v);
  k_lr_final<<<(int)std::min<int64_t>((d.ucols + 7) / 8, 4096), 256, 0, st>>>(d, quad);
  if (quad) k_lr_quad<<<1, 1024, 0, st>>>(d);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ setup

// diag(H)_j = h0_j + sum_i w_R,i R_ij^2 + sum_r uw_r U_jr^2 + Hs_jj  (computed once; Section
// 4.1.2 caches it).
__global__ void k_diagH(Dev d) {
  for (int64_t j = gwarp(); j < d.n; j += nwarps()) {
    double acc = warp_row_dot<true>(d.RT_ptr[j], d.RT_ptr[j + 1], d.RT_idx, d.RT_val, d.wR);
    if (d.ucols) {
      double ul = 0.0;
      for (int64_t r = threadIdx.x & 31; r < d.ucols; r += 32) {
        const double u = d.U[j * d.ucols + r];
        ul = fma(d.uw[r] * u, u, ul);
      }
      acc += warp_sum(ul);
    }
    double hjj = 0.0;
    if (d.Hs_ptr) {
      for (int64_t e = d.Hs_ptr[j] + (threadIdx.x & 31); e < d.Hs_ptr[j + 1]; e += 32)
        if (d.Hs_idx[e] == j) hjj += d.Hs_val[e];
      hjj = warp_sum(hjj);
    }
    if ((threadIdx.x & 31) == 0) d.diagH[j] = d.h0[j] + acc + hjj;
  }
}

__global__ void k_fill_rowk(Dev d) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d.nR; r += (int64_t)gridDim.x * blockDim.x)
    d.rowk[r] = -1;
}

__global__ void k_fill_rowk2(Dev d) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.m; k += (int64_t)gridDim.x * blockDim.x)
    d.rowk[d.arow[k]] = (int32_t)k;
}

// rowk: the constraint index of each row of R (-1 for rows of the factor alone).
cudaError_t launch_fill_rowk(const Dev& d, cudaStream_t st) {
  if (!d.nR) return cudaSuccess;
  const int b = (int)std::min<int64_t>((d.nR + kBlock - 1) / kBlock, 4096);
  k_fill_rowk<<<b, kBlock, 0, st>>>(d);
  if (d.m) k_fill_rowk2<<<(int)std::min<int64_t>((d.m + kBlock - 1) / kBlock, 4096), kBlock, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_diagH(const Dev& d, cudaStream_t st) {
  Geo g = make_geo(d);
  if (g.gN) k_diagH<<<g.gN, kBlock, 0, st>>>(d);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ residuals

// t = R x; v = w_R o t; partial sum of w_R t^2 (the factor part of x^T H x).
template <int G>
__global__ void k_rows_resid(Dev d, double* part) {
  __shared__ double sh[32];
  double acc = 0.0;
  FOR_GROUP_ROWS(G, r, ok, d.nR) {
    const int64_t beg = ok ? d.R_ptr[r] : 0, end = ok ? d.R_ptr[r + 1] : 0;
    const double t = group_row_dot<G, false>(beg, end, glane<G>(), d.R_idx, d.R_val, d.x);
    if (ok && glane<G>() == 0) {
      const double w = d.wR[r];
      d.tR[r] = t;
      d.vR[r] = w * t;
      acc = fma(w * t, t, acc);
    }
  }
  acc = block_reduce<0>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// Constraint rows: r_p = A x + s - b, r_s = s o y - mu, and y placed on R rows (vR2).
__global__ void k_cons_resid(Dev d, double* part) {
  __shared__ double sh[32];
  const double mu = d.sc->mu;
  double rp_inf = 0.0, viol = 0.0, rs_inf = 0.0, by = 0.0, sy = 0.0, ymax = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.m; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t row = d.arow[k];
    const double ax = d.tR[row];
    const double rp = ax + d.s[k] - d.b[k];
    const double rs = d.s[k] * d.y[k] - mu;
    d.rp[k] = rp;
    d.vR2[row] = d.y[k];
    rp_inf = fmax(rp_inf, fabs(rp));
    viol = fmax(viol, ax - d.b[k]);
    rs_inf = fmax(rs_inf, fabs(rs));
    by = fma(d.b[k], d.y[k], by);
    ymax = fmax(ymax, fabs(d.y[k]));
    sy = fma(d.s[k], d.y[k], sy);
  }
  const int K = kMaxRedBlocks;
  double v;
  v = block_reduce<1>(rp_inf, sh); if (threadIdx.x == 0) part[1 * K + blockIdx.x] = v;
  v = block_reduce<1>(viol, sh);   if (threadIdx.x == 0) part[2 * K + blockIdx.x] = v;
  v = block_reduce<1>(rs_inf, sh); if (threadIdx.x == 0) part[3 * K + blockIdx.x] = v;
  v = block_reduce<0>(by, sh);     if (threadIdx.x == 0) part[4 * K + blockIdx.x] = v;
  v = block_reduce<0>(sy, sh);     if (threadIdx.x == 0) part[5 * K + blockIdx.x] = v;
  v = block_reduce<1>(ymax, sh);   if (threadIdx.x == 0) part[28 * K + blockIdx.x] = v;
}

// Variables: Hx = R^T vR + Hs x + h0 o x, A^T y (over the stored A^T, y placed on R rows in
// vR2), r_d, r_l, r_u and the scalar parts
// of the objective, the dual objective and the complementarity sum.
template <int G>
__global__ void __launch_bounds__(256, 4) k_cols_resid(Dev d, double* part) {
  __shared__ double sh[32];
  const double mu = d.sc->mu;
  double rd_inf = 0.0, hx_inf = 0.0, aty_inf = 0.0, rc_inf = 0.0, xHsx = 0.0, cx = 0.0, lzl = 0.0,
         uzu = 0.0, tz = 0.0, bviol = 0.0, cert = 0.0, zmax = 0.0;
  FOR_GROUP_ROWS(G, j, ok, d.n) {
    const int64_t beg = ok ? d.RT_ptr[j] : 0, end = ok ? d.RT_ptr[j + 1] : 0;
    const double hx_f = group_row_dot<G, false>(beg, end, glane<G>(), d.RT_idx, d.RT_val, d.vR);
    const int64_t ab = ok ? d.AT_ptr[j] : 0, ae = ok ? d.AT_ptr[j + 1] : 0;
    const double aty = group_row_dot<G, false>(ab, ae, glane<G>(), d.AT_idx, d.AT_val, d.vR2);
    double hs = 0.0;
    if (d.Hs_ptr) {
      const int64_t hb = ok ? d.Hs_ptr[j] : 0, he = ok ? d.Hs_ptr[j + 1] : 0;
      hs = group_row_dot<G, false>(hb, he, glane<G>(), d.Hs_idx, d.Hs_val, d.x);
    }
    const double lr = d.ucols ? lr_row<G>(d, j, ok, glane<G>()) : 0.0;
    if (ok && glane<G>() == 0) {
      const double xj = d.x[j];
      const double hsx = hs + d.h0[j] * xj;
      const double hx = hx_f + hsx + lr;
      const double zl = d.zl[j], zu = d.zu[j];
      const double rd = hx + d.c[j] + aty - zl + zu;
      d.Hx[j] = hx;
      d.Aty[j] = aty;
      d.rd[j] = rd;
      cert = fmax(cert, fabs(aty - zl + zu));
      zmax = fmax(zmax, fmax(fabs(zl), fabs(zu)));
      rd_inf = fmax(rd_inf, fabs(rd));
      hx_inf = fmax(hx_inf, fabs(hx));
      aty_inf = fmax(aty_inf, fabs(aty));
      xHsx = fma(xj, hsx, xHsx);
      cx = fma(d.c[j], xj, cx);
      if (d.fl[j]) {
        const double tl = xj - d.l[j];
        rc_inf = fmax(rc_inf, fabs(tl * zl - mu));
        lzl = fma(d.l[j], zl, lzl);
        tz = fma(tl, zl, tz);
        bviol = fmax(bviol, -tl);
      }
      if (d.fu[j]) {
        const double tu = d.u[j] - xj;
        rc_inf = fmax(rc_inf, fabs(tu * zu - mu));
        uzu = fma(d.u[j], zu, uzu);
        tz = fma(tu, zu, tz);
        bviol = fmax(bviol, -tu);
      }
    }
  }
  const int K = kMaxRedBlocks;
  double v;
  v = block_reduce<1>(rd_inf, sh);  if (threadIdx.x == 0) part[6 * K + blockIdx.x] = v;
  v = block_reduce<1>(hx_inf, sh);  if (threadIdx.x == 0) part[7 * K + blockIdx.x] = v;
  v = block_reduce<1>(aty_inf, sh); if (threadIdx.x == 0) part[8 * K + blockIdx.x] = v;
  v = block_reduce<1>(rc_inf, sh);  if (threadIdx.x == 0) part[9 * K + blockIdx.x] = v;
  v = block_reduce<0>(xHsx, sh);    if (threadIdx.x == 0) part[10 * K + blockIdx.x] = v;
  v = block_reduce<0>(cx, sh);      if (threadIdx.x == 0) part[11 * K + blockIdx.x] = v;
  v = block_reduce<0>(lzl, sh);     if (threadIdx.x == 0) part[12 * K + blockIdx.x] = v;
  v = block_reduce<0>(uzu, sh);     if (threadIdx.x == 0) part[13 * K + blockIdx.x] = v;
  v = block_reduce<0>(tz, sh);      if (threadIdx.x == 0) part[14 * K + blockIdx.x] = v;
  v = block_reduce<1>(bviol, sh);   if (threadIdx.x == 0) part[15 * K + blockIdx.x] = v;
  v = block_reduce<1>(cert, sh);    if (threadIdx.x == 0) part[29 * K + blockIdx.x] = v;
  v = block_reduce<1>(zmax, sh);    if (threadIdx.x == 0) part[30 * K + blockIdx.x] = v;
}

// One block: totals of the partials, then the relative KKT residual (primal, dual, gap), the
// objective values and the norm of the mu test.
//   primal = max(viol_A, viol_bounds) / (1 + ||b||), dual = ||r_d|| / (1 + max(||c||, ||Hx||, ||A^T y||)),
//   gap = |pobj - dobj| / (1 + |pobj| + |dobj|),
//   ||r||_mu = max(||r_s, r_l, r_u||, (1 + |pobj|) / N_c * max(||r_p|| / (1 + ||b||), ||r_d|| / (1 + ||c||))).
__global__ void k_resid_final(Dev d, int gR, int gM, int gN, const double* part) {
  // all 19 block partials reduced in one pass: per thread over its blocks, then per warp by
  // shuffles, then across warps (fixed order); sums (op 0) and maxima (op 1)
  constexpr int NQ = 19;
  const int slot[NQ] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 28, 29, 30};
  const int opq[NQ] = {0, 1, 1, 1, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 0, 1, 1, 1, 1};
  const int nbq[NQ] = {gR, gM, gM, gM, gM, gM, gN, gN, gN, gN, gN, gN, gN, gN, gN, gN, gM, gN, gN};
  __shared__ double red[32][NQ];
  __shared__ double res[NQ];
  const int K = kMaxRedBlocks;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    acc[q] = opq[q] == 0 ? 0.0 : -INFINITY;
    for (int b = threadIdx.x; b < nbq[q]; b += blockDim.x) {
      const double v = part[slot[q] * K + b];
      acc[q] = opq[q] == 0 ? acc[q] + v : fmax(acc[q], v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, acc[q], o);
      acc[q] = opq[q] == 0 ? acc[q] + w : fmax(acc[q], w);
    }
    if (lane == 0) red[warp][q] = acc[q];
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    const int q = threadIdx.x;
    double t = opq[q] == 0 ? 0.0 : -INFINITY;
    for (int w = 0; w < nw; ++w) t = opq[q] == 0 ? t + red[w][q] : fmax(t, red[w][q]);
    res[q] = t;
  }
  __syncthreads();
  const double xFx = res[0];
  const double rp_inf = fmax(0.0, res[1]);
  const double viol_a = fmax(0.0, res[2]);
  const double rs_inf = fmax(0.0, res[3]);
  const double by = res[4];
  const double sy = res[5];
  const double rd_inf = fmax(0.0, res[6]);
  const double hx_inf = fmax(0.0, res[7]);
  const double aty_inf = fmax(0.0, res[8]);
  const double rc_inf = fmax(0.0, res[9]);
  const double xHsx = res[10];
  const double cx = res[11];
  const double lzl = res[12];
  const double uzu = res[13];
  const double tz = res[14];
  const double viol_b = fmax(0.0, res[15]);
  const double ymax = d.m ? fmax(0.0, res[16]) : 0.0;
  const double cert = fmax(0.0, res[17]);
  const double zmax = fmax(0.0, res[18]);
  if (threadIdx.x == 0) {
    Scal* sc = d.sc;
    const double xHx = xFx + xHsx + (d.ucols ? sc->lr_quad : 0.0);
    const double pobj = 0.5 * xHx + cx;
    const double dobj = -0.5 * xHx - by + lzl - uzu;
    const double bn = sc->bnorm, cn = sc->cnorm;
    const double primal = fmax(viol_a, viol_b) / (1.0 + bn);
    const double dual = rd_inf / (1.0 + fmax(cn, fmax(hx_inf, aty_inf)));
    const double gap = fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
    sc->res_primal = primal;
    sc->res_dual = dual;
    sc->res_gap = gap;
    double rk = fmax(primal, fmax(dual, gap));
    if (!isfinite(rk)) rk = INFINITY;
    sc->rel_kkt = rk;
    sc->pobj = pobj;
    sc->dobj = dobj;
    sc->rp_inf = rp_inf;
    sc->rd_inf = rd_inf;
    sc->rc_inf = fmax(rs_inf, rc_inf);
    const int nc = sc->ncomp > 0 ? sc->ncomp : 1;
    const double ep = rp_inf / (1.0 + bn), ed = rd_inf / (1.0 + cn);
    sc->rnorm_mu = fmax(fmax(rs_inf, rc_inf), (1.0 + fabs(pobj)) / nc * fmax(ep, ed));
    sc->comp_mean = (sy + tz) / nc;
    const double mi = fmax(ymax, zmax);
    sc->mult_inf = mi;
    sc->cert_res = mi > 0.0 ? cert / mi : INFINITY;
    sc->cert_gap = mi > 0.0 ? (by - lzl + uzu) / mi : 0.0;
  }
}

cudaError_t launch_residual_summary(const Dev& d, const Geo& g, cudaStream_t st) {
  double* part = d.partials;
  if (d.nR) {
    cudaMemsetAsync(d.vR2, 0, sizeof(double) * d.nR, st);
    DISPATCH_G(d.g_rows, k_rows_resid<G><<<g.gR, kBlock, 0, st>>>(d, part));
  }
  if (d.m) k_cons_resid<<<g.eM, kBlock, 0, st>>>(d, part);
  launch_lr(d, d.x, 1, st);
  DISPATCH_G(d.g_cols, k_cols_resid<G><<<g.gNr, kBlock, 0, st>>>(d, part));
  k_resid_final<<<1, 512, 0, st>>>(d, g.gR, g.eM, g.gNr, part);
  return cudaGetLastError();
}

// Complementarity residuals as vectors (for the step-level query): r_s into ds, r_l into dzl,
// r_u into dzu.
__global__ void k_comp_resid(Dev d) {
  const double mu = d.sc->mu;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.m; k += (int64_t)gridDim.x * blockDim.x)
    d.ds[k] = d.s[k] * d.y[k] - mu;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    d.dzl[j] = d.fl[j] ? (d.x[j] - d.l[j]) * d.zl[j] - mu : 0.0;
    d.dzu[j] = d.fu[j] ? (d.u[j] - d.x[j]) * d.zu[j] - mu : 0.0;
  }
}

cudaError_t launch_comp_resid(const Dev& d, const Geo& g, cudaStream_t st) {
  k_comp_resid<<<std::max(g.eN, g.eM), kBlock, 0, st>>>(d);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ start point

static __device__ void set_eta(Scal* sc);

// x0 = 0 projected into the box shrunk by delta_j = 0.1 min(1, (u_j - l_j) / 2) (0.1 for a
// one-sided bound; 0 for a free variable).
__global__ void k_start_x(Dev d) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    const bool fl = d.fl[j], fu = d.fu[j];
    const double width = (fl && fu) ? d.u[j] - d.l[j] : 2.0;
    const double delta = 0.1 * fmin(1.0, 0.5 * width);
    double x = 0.0;
    if (fl) x = fmax(x, d.l[j] + delta);
    if (fu) x = fmin(x, d.u[j] - delta);
    d.x[j] = x;
  }
}

// s0 = max(b - A x0, 1)   (tR holds R x0)
__global__ void k_start_s(Dev d) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.m; k += (int64_t)gridDim.x * blockDim.x)
    d.s[k] = fmax(d.b[k] - d.tR[d.arow[k]], 1.0);
}

// g = H x0 + c; z_l0 = max(1, g), z_u0 = max(1, -g) on finite bounds.
template <int G>
__global__ void k_start_z(Dev d) {
  FOR_GROUP_ROWS(G, j, ok, d.n) {
    const int64_t beg = ok ? d.RT_ptr[j] : 0, end = ok ? d.RT_ptr[j + 1] : 0;
    const double hx = group_row_dot<G, false>(beg, end, glane<G>(), d.RT_idx, d.RT_val, d.vR);
    double hs = 0.0;
    if (d.Hs_ptr) {
      const int64_t hb = ok ? d.Hs_ptr[j] : 0, he = ok ? d.Hs_ptr[j + 1] : 0;
      hs = group_row_dot<G, false>(hb, he, glane<G>(), d.Hs_idx, d.Hs_val, d.x);
    }
    if (d.ucols) hs += lr_row<G>(d, j, ok, glane<G>());
    if (ok && glane<G>() == 0) {
      const double g = hx + hs + d.h0[j] * d.x[j] + d.c[j];
      d.zl[j] = d.fl[j] ? fmax(1.0, g) : 0.0;
      d.zu[j] = d.fu[j] ? fmax(1.0, -g) : 0.0;
    }
  }
}

// y0 = 1 on every row (theta starts moderate: no constraint row begins stiff).
__global__ void k_start_y(Dev d) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.m; k += (int64_t)gridDim.x * blockDim.x)
    d.y[k] = 1.0;
}

__global__ void k_start_mu(Dev d) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    Scal* sc = d.sc;
    sc->mu0 = sc->comp_mean > 0.0 ? sc->comp_mean : 1.0;
    sc->mu0_cold = sc->mu0;
    sc->mu = sc->mu0;
    sc->ipm_iter = 0;
    sc->stop = 0;
    sc->status = DS_RUNNING;
    set_eta(sc);
  }
}

cudaError_t launch_start_point(const Dev& d, const Geo& g, cudaStream_t st) {
  k_start_x<<<g.eN, kBlock, 0, st>>>(d);
  if (d.nR) DISPATCH_G(d.g_rows, k_rows_resid<G><<<g.gR, kBlock, 0, st>>>(d, d.partials));
  if (d.m) k_start_s<<<g.eM, kBlock, 0, st>>>(d);
  launch_lr(d, d.x, 0, st);
  DISPATCH_G(d.g_cols, k_start_z<G><<<g.gN, kBlock, 0, st>>>(d));
  if (d.m) k_start_y<<<g.eM, kBlock, 0, st>>>(d);
  cudaError_t e = launch_residual_summary(d, g, st);
  if (e != cudaSuccess) return e;
  k_start_mu<<<1, 32, 0, st>>>(d);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ control

// Inexact-Newton forcing term of the PCG solve: ||r|| <= eta ||rhs|| with
// eta = clamp(eta_factor * relKKT, eta_min, eta_max) (reading; the paper states no tolerance).
static __device__ void set_eta(Scal* sc) {
  if (sc->eta_override) return;
  double e = sc->eta_factor * sc->rel_kkt;
  if (!(e <= sc->eta_max)) e = sc->eta_max;
  if (e < sc->eta_min) e = sc->eta_min;
  sc->eta = e;
}

// Algorithm 1's tail on the device: stop when rel KKT <= tol (reading of "mu <= mu_tol"),
// else mu <- mu / 10 when ||r|| < mu; then the PCG tolerance eta for the next Newton step.
__global__ void k_control(Dev d, cudaGraphConditionalHandle h, int set_cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Scal* sc = d.sc;
  sc->ipm_iter += 1;
  const double rk = sc->rel_kkt;
  const double mu_step = sc->mu;
  const int refine = d.storage != ST_F64 ? sc->refine_it : 0;
  sc->cg_total += sc->cg_iter;
  sc->refine_total += refine;
  if (sc->cg_iter > sc->max_cg_step) sc->max_cg_step = sc->cg_iter;
  // PCG stall: the PCG of two consecutive Newton steps ended at the iteration limit with a
  // residual above 1e-2 of its right-hand side (worse than the loosest tolerance the method
  // asks for).  A direction that misses a tight tolerance but is otherwise accurate is kept
  // (inexact Newton): the paper's doubly augmented system under Jacobi PCG lives there.
  const double cg_rel = sc->rhs2 > 0.0 ? sqrt(sc->rr / sc->rhs2) : 0.0;
  sc->cg_fail_run = (sc->cg_conv || cg_rel <= 1e-2) ? 0 : sc->cg_fail_run + 1;
  if (sc->status == DS_RUNNING && sc->cg_fail_run >= 2) sc->status = DS_CG_STALL;
  if (sc->status == DS_NUMERICAL || sc->status == DS_CG_STALL || sc->status == DS_TIMEOUT) {
    sc->stop = 1;
  } else if (sc->ipm_iter >= 5 && !(sc->res_primal <= sc->tol_kkt) && sc->mult_inf > 1e10 &&
             isfinite(sc->mult_inf) && sc->cert_res <= 1e-8 && sc->cert_gap < -1e-8) {
    // the multipliers diverge along a Farkas certificate of primal infeasibility:
    // y >= 0, z >= 0 with A^T y - z_l + z_u ~ 0 and b^T y - l^T z_l + u^T z_u < 0
    sc->stop = 1;
    sc->status = DS_INFEASIBLE;
  } else if (!isfinite(rk) || !isfinite(sc->pobj)) {
    sc->stop = 1;
    sc->status = DS_NUMERICAL;
  } else if (rk <= sc->tol_kkt) {
    sc->stop = 1;
    sc->status = DS_OK;
  } else if (sc->ipm_iter >= sc->max_ipm) {
    sc->stop = 1;
    sc->status = DS_MAX_ITER;
  } else if (sc->rnorm_mu < sc->mu) {
    sc->mu = fmax(sc->mu * 0.1, sc->mu0 * 1e-16);
  }
  set_eta(sc);
  if (d.trace && sc->trace_rows < sc->trace_cap) {
    double* t = d.trace + (int64_t)sc->trace_rows * kTraceCols;
    t[0] = sc->ipm_iter; t[1] = mu_step; t[2] = rk; t[3] = sc->res_primal; t[4] = sc->res_dual;
    t[5] = sc->res_gap; t[6] = sc->alpha_p; t[7] = sc->alpha_d; t[8] = sc->cg_iter; t[9] = sc->cg_conv;
    t[10] = sc->n_stiff; t[11] = sc->rhs2 > 0 ? sqrt(sc->rr / sc->rhs2) : 0.0; t[12] = sc->eta_used; t[13] = refine;
    sc->trace_rows += 1;
  }
  if (set_cond) cudaGraphSetConditional(h, sc->stop ? 0u : 1u);
}

cudaError_t launch_control(const Dev& d, cudaStream_t st, cudaGraphConditionalHandle h) {
  k_control<<<1, 32, 0, st>>>(d, h, h != 0 ? 1 : 0);
  return cudaGetLastError();
}

// Start of a solve on the device: per-solve totals and the trace cleared.
__global__ void k_solve_begin(Dev d) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Scal* sc = d.sc;
  sc->cg_total = 0;
  sc->refine_total = 0;
  sc->max_cg_step = 0;
  sc->trace_rows = 0;
  sc->max_stiff_seen = 0;
  sc->fallback_total = 0;
  sc->cg_fail_run = 0;
  sc->stop = 0;
  sc->status = DS_RUNNING;
}

cudaError_t launch_solve_begin(const Dev& d, cudaStream_t st) {
  k_solve_begin<<<1, 32, 0, st>>>(d);
  return cudaGetLastError();
}

// Warm start from the current iterate: mu0 = its complementarity mean (after a residual summary).
__global__ void k_warm_mu(Dev d) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Scal* sc = d.sc;
  sc->mu0 = sc->comp_mean > 0.0 ? sc->comp_mean : 1.0;
  sc->mu = sc->mu0;
  sc->ipm_iter = 0;
  set_eta(sc);
}

// Warm start (reading; the paper warm-starts the SQP's QPs, Section 3.2, without a recipe):
// every complementarity pair of the previous solution is raised to at least
// mu_w = warm_rho * mu0_cold (mu0 of the last cold start on this handle): s and y scaled
// together by sqrt(mu_w / (s y)), z_l, z_u raised to mu_w / t.  No shift before a cold start.
__global__ void k_warm_shift(Dev d) {
  const double muw = d.sc->warm_rho * d.sc->mu0_cold;
  if (!(muw > 0.0)) return;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.m; k += (int64_t)gridDim.x * blockDim.x) {
    const double sy = d.s[k] * d.y[k];
    if (sy < muw) {
      const double f = sqrt(muw / fmax(sy, 1e-300));
      d.s[k] *= f;
      d.y[k] *= f;
    }
  }
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    if (d.fl[j]) d.zl[j] = fmax(d.zl[j], muw / (d.x[j] - d.l[j]));
    if (d.fu[j]) d.zu[j] = fmax(d.zu[j], muw / (d.u[j] - d.x[j]));
  }
}

cudaError_t launch_warm_start(const Dev& d, const Geo& g, cudaStream_t st) {
  k_warm_shift<<<std::max(g.eN, g.eM), kBlock, 0, st>>>(d);
  cudaError_t e = launch_residual_summary(d, g, st);
  if (e != cudaSuccess) return e;
  k_warm_mu<<<1, 32, 0, st>>>(d);
  return cudaGetLastError();
}

__global__ void k_set_cond(cudaGraphConditionalHandle h, unsigned v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, v);
}

cudaError_t launch_set_cond(cudaGraphConditionalHandle h, unsigned v, cudaStream_t st) {
  k_set_cond<<<1, 32, 0, st>>>(h, v);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ diagonal update

// theta = y / s; omega = w_R + theta on the constraint rows (omega preset to w_R); twice
// theta for the doubly augmented system.
__global__ void k_diag_m(Dev d) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.m; k += (int64_t)gridDim.x * blockDim.x) {
    const double th = d.y[k] / d.s[k];
    const int32_t row = d.arow[k];
    d.theta[k] = th;
    // doubly augmented system: its (1,1) block carries 2 B^T D^-1 B = 2 A^T Theta A
    const double thf = d.aug ? 2.0 * th : th;
    d.omega[row] = d.wR[row] + thf;
    d.thR[row] = thf;
  }
}

// sigma = z_l / t_l + z_u / t_u; M0 = diag(H) + sigma.
__global__ void k_diag_n(Dev d) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    double sg = 0.0;
    if (d.fl[j]) sg += d.zl[j] / (d.x[j] - d.l[j]);
    if (d.fu[j]) sg += d.zu[j] / (d.u[j] - d.x[j]);
    d.sigma[j] = sg;
    const double m0 = d.diagH[j] + sg;
    d.M0[j] = m0;
    d.Minv[j] = 1.0 / m0;   // 1 / M0 until the Jacobi diagonal of the moderate rows replaces it
  }
}

cudaError_t launch_diag_update(const Dev& d, const Geo& g, cudaStream_t st) {
  if (d.nR) {
    cudaMemcpyAsync(d.omega, d.wR, sizeof(double) * d.nR, cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(d.thR, 0, sizeof(double) * d.nR, st);
  }
  if (d.m) k_diag_m<<<g.eM, kBlock, 0, st>>>(d);
  k_diag_n<<<g.eN, kBlock, 0, st>>>(d);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ Jacobi

// M_j = M0_j + sum_k A_kj^2 thR_k  (thR: theta of the constraint rows kept in the diagonal part;
// the factor rows' part w_R is already in M0 through diag(H)).
// Writes 1 / M_j to out (INV) or M_j.
template <bool INV, int G>
__global__ void k_jacobi(Dev d, double* out) {
  FOR_GROUP_ROWS(G, j, ok, d.n) {
    const int64_t beg = ok ? d.AT_ptr[j] : 0, end = ok ? d.AT_ptr[j + 1] : 0;
    const double a = group_row_dot<G, true>(beg, end, glane<G>(), d.AT_idx, d.AT_val, d.thR);
    if (ok && glane<G>() == 0) {
      const double mj = d.M0[j] + a;
      out[j] = INV ? 1.0 / mj : mj;
    }
  }
}

cudaError_t launch_jacobi_full(const Dev& d, const Geo& g, double* out, cudaStream_t st) {
  DISPATCH_G(d.g_at, k_jacobi<false, G><<<g.gN, kBlock, 0, st>>>(d, out));
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ stiff rows

// ratio_k = theta_k sum_j A_kj^2 / M0_j; histogram of log2(ratio / gamma) in half-octave bins;
// the last block picks the smallest threshold bin whose cumulative count from the top stays
// <= stiff_max.  Rows with ratio >= stiff_thresh form the low-rank correction.
template <int G>
__global__ void k_stiff_ratio(Dev d) {
  __shared__ unsigned int h[kHistBins];
  __shared__ bool s_last;
  for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const double gamma = d.sc->stiff_gamma;
  FOR_GROUP_ROWS(G, k, ok, d.m) {
    const int32_t row = ok ? d.arow[k] : 0;
    const int64_t beg = ok ? d.R_ptr[row] : 0, end = ok ? d.R_ptr[row + 1] : 0;
    // sum_j R_kj^2 / M0_j with 1 / M0 precomputed in Minv
    const double acc = group_row_dot<G, true>(beg, end, glane<G>(), d.R_idx, d.R_val, d.Minv);
    if (ok && glane<G>() == 0) {
      const double ratio = d.theta[k] * acc;
      d.ratio[k] = ratio;
      if (ratio > gamma) {
        int bin = (int)floor(2.0 * log2(ratio / gamma));
        bin = bin < 0 ? 0 : (bin >= kHistBins ? kHistBins - 1 : bin);
        atomicAdd(&h[bin], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kHistBins; i += blockDim.x)
    if (h[i]) atomicAdd(&d.hist[i], h[i]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(&d.sc->ticket[T_HIST], 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    const int cap = d.sc->stiff_max;
    unsigned int cum = 0;
    int cut = kHistBins;  // no stiff rows
    for (int b = kHistBins - 1; b >= 0; --b) {
      unsigned int c = __ldcg(&d.hist[b]);
      if (cum + c > (unsigned)cap) break;
      cum += c;
      cut = b;
    }
    // rows in bins >= cut are stiff: threshold = gamma * 2^(cut/2) (bins are half octaves)
    d.sc->stiff_thresh = cut >= kHistBins ? INFINITY : (cut == 0 ? gamma : gamma * exp2(0.5 * cut));
    for (int b = 0; b < kHistBins; ++b) d.hist[b] = 0u;
    d.sc->ticket[T_HIST] = 0u;
  }
}

// Exclusive scan of per-item 0/1 (or counts) by one block in two levels: every thread scans
// a contiguous run serially, then the block scans the run totals.  Returns the total; calls
// emit(i, offset) for every item i in order-preserving positions.
template <typename Val, typename Emit>
__device__ long long block_scan_runs(int64_t count, Val val, Emit emit) {
  __shared__ long long tsum[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  const int64_t run = (count + nt - 1) / nt;
  const int64_t b0 = t * run, b1 = b0 + run < count ? b0 + run : count;
  long long acc = 0;
  for (int64_t i = b0; i < b1; ++i) acc += val(i);
  tsum[t] = acc;
  __syncthreads();
  // Hillis-Steele inclusive scan of the nt run totals
  for (int off = 1; off < nt; off <<= 1) {
    long long v = t >= off ? tsum[t - off] : 0;
    __syncthreads();
    tsum[t] += v;
    __syncthreads();
  }
  long long base = t ? tsum[t - 1] : 0;
  const long long total = tsum[nt - 1];
  for (int64_t i = b0; i < b1; ++i) {
    const long long v = val(i);
    emit(i, base, v);
    base += v;
  }
  __syncthreads();
  return total;
}

// Ordered compaction (one block): slot of every stiff row, thR = 0 on stiff rows.
__global__ void k_stiff_compact(Dev d) {
  const double thr = d.sc->stiff_thresh;
  const double gamma = d.sc->stiff_gamma;
  const int cap = d.stiff_cap;
  auto flag = [&](int64_t k) -> long long {
    const double rt = d.ratio[k];
    return (rt > gamma && rt >= thr) ? 1 : 0;
  };
  const long long total = block_scan_runs(d.m, flag, [&](int64_t k, long long off, long long v) {
    const int32_t row = d.arow[k];
    if (v && off < cap) {
      d.stiff_k[off] = (int32_t)k;
      d.slotR[row] = (int32_t)off;
      d.thR[row] = 0.0;
    } else {
      d.slotR[row] = -1;
    }
  });
  if (threadIdx.x == 0) {
    const int ns = total < cap ? (int)total : cap;
    d.sc->n_stiff = ns;
    if (ns > d.sc->max_stiff_seen) d.sc->max_stiff_seen = ns;
  }
}

// Stiff entries per variable (count, then ordered fill) from the stored transpose.
__global__ void k_sc_count(Dev d) {
  if (d.sc->n_stiff == 0) return;
  for (int64_t j = gwarp(); j < d.n; j += nwarps()) {
    int cnt = 0;
    for (int64_t e = d.AT_ptr[j] + (threadIdx.x & 31); e < d.AT_ptr[j + 1]; e += 32)
      cnt += d.slotR[d.AT_idx[e]] >= 0 ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) d.sc_cnt[j] = cnt;
  }
}

// Exclusive scan of sc_cnt into sc_ptr (one block, two levels).
__global__ void k_sc_scan(Dev d) {
  if (d.sc->n_stiff == 0) return;
  const long long total = block_scan_runs(d.n, [&](int64_t j) -> long long { return d.sc_cnt[j]; },
                                          [&](int64_t j, long long off, long long) { d.sc_ptr[j] = off; });
  if (threadIdx.x == 0) {
    d.sc_ptr[d.n] = total;
    if (total > d.sc_cap) d.sc->n_stiff = 0;   // does not fit: fall back to plain Jacobi
  }
}

__global__ void k_sc_fill(Dev d) {
  if (d.sc->n_stiff == 0) return;
  const int lane = threadIdx.x & 31;
  for (int64_t j = gwarp(); j < d.n; j += nwarps()) {
    int64_t out = d.sc_ptr[j];
    for (int64_t e0 = d.AT_ptr[j]; e0 < d.AT_ptr[j + 1]; e0 += 32) {
      const int64_t e = e0 + lane;
      int slot = -1;
      if (e < d.AT_ptr[j + 1]) slot = d.slotR[d.AT_idx[e]];
      const unsigned bal = __ballot_sync(0xffffffffu, slot >= 0);
      if (slot >= 0) {
        const int64_t pos = out + __popc(bal & ((1u << lane) - 1u));
        d.sc_slot[pos] = slot;
        d.sc_val[pos] = d.AT_val[e];
      }
      out += __popc(bal);
    }
  }
}

// G = Theta_s^{-1} + A_s M^{-1} A_s^T (dense, n_stiff x n_stiff, leading dimension stiff_cap).
// One block per stiff row a accumulates row a in shared memory: for every entry (j, R_aj) of
// the row, add R_aj / M_j * (column j's stiff entries).  Entries of a column list are distinct
// slots, so lanes never collide; the j order is fixed, hence deterministic.
__global__ void k_gram_G(Dev d) {
  extern __shared__ double grow[];
  const int ns = d.sc->n_stiff;
  const int cap = d.stiff_cap;
  for (int a = blockIdx.x; a < ns; a += gridDim.x) {
    for (int i = threadIdx.x; i < ns; i += blockDim.x) grow[i] = 0.0;
    __syncthreads();
    const int32_t k = d.stiff_k[a];
    const int32_t row = d.arow[k];
    for (int64_t e = d.R_ptr[row]; e < d.R_ptr[row + 1]; ++e) {
      const int32_t j = d.R_idx[e];
      const double f = d.R_val[e] * d.Minv[j];
      const int64_t b0 = d.sc_ptr[j], b1 = d.sc_ptr[j + 1];
      for (int64_t t = b0 + threadIdx.x; t < b1; t += blockDim.x) grow[d.sc_slot[t]] += f * d.sc_val[t];
      __syncthreads();
    }
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
      double v = grow[i];
      if (i == a) v += 1.0 / d.theta[k];
      d.G[(int64_t)a * cap + i] = v;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------ rhs

// u = theta o r_p - r_s / s placed on R rows (vR2, pre-zeroed); the doubly augmented system
// takes 2u there and its bottom block's right-hand side, start and Jacobi diagonal.
__global__ void k_rhs_m(Dev d) {
  const double mu = d.sc->mu;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.m; k += (int64_t)gridDim.x * blockDim.x) {
    const double s = d.s[k];
    const double rs = s * d.y[k] - mu;
    const double u = d.theta[k] * d.rp[k] - rs / s;   // theta o r2, r2 = r_p - r_s / y
    if (d.aug) {
      // eq:2x2_augmented: top r1 + 2 B^T D^-1 r2 = r1 - 2 A^T (theta o r2); bottom r2;
      // Jacobi on the bottom block D = s / y: 1 / D = theta
      const double r2 = d.rp[k] - rs / d.y[k];
      d.vR2[d.arow[k]] = 2.0 * u;
      d.rhs[d.n + k] = r2;
      d.r[d.n + k] = r2;
      d.dx[d.n + k] = 0.0;
      d.Minv[d.n + k] = d.theta[k];
    } else {
      d.vR2[d.arow[k]] = u;
    }
  }
}

// PCG start from ||rhs||^2: tolerance eta^2 ||rhs||^2, counters reset.
static __device__ void finish_rhs(Scal* sc, double rhs2) {
  sc->rhs2 = rhs2;
  sc->eta_used = sc->eta;
  sc->tol2 = sc->eta * sc->eta * rhs2;
  sc->cg_iter = 0;
  sc->cg_conv = 0;
  sc->cg_done = (rhs2 == 0.0 || !isfinite(rhs2)) ? 1 : 0;
  if (!isfinite(rhs2)) sc->status = DS_NUMERICAL;
  else if (rhs2 == 0.0) sc->cg_conv = 1;
}

// rhs = -r_d - r_l / t_l + r_u / t_u - A^T u (u = vR2 on the constraint rows); PCG start
// r = rhs, dx = 0; ||rhs||^2.
template <int G>
__global__ void k_rhs_n(Dev d) {
  __shared__ double sh[32];
  const double mu = d.sc->mu;
  double r2 = 0.0;
  FOR_GROUP_ROWS(G, j, ok, d.n) {
    const int64_t beg = ok ? d.AT_ptr[j] : 0, end = ok ? d.AT_ptr[j + 1] : 0;
    const double atu = group_row_dot<G, false>(beg, end, glane<G>(), d.AT_idx, d.AT_val, d.vR2);
    if (ok && glane<G>() == 0) {
      double g = -d.rd[j] - atu;
      const double xj = d.x[j];
      if (d.fl[j]) { const double tl = xj - d.l[j]; g -= (tl * d.zl[j] - mu) / tl; }
      if (d.fu[j]) { const double tu = d.u[j] - xj; g += (tu * d.zu[j] - mu) / tu; }
      d.rhs[j] = g;
      d.r[j] = g;
      d.dx[j] = 0.0;
      r2 = fma(g, g, r2);
    }
  }
  double v[1] = {r2};
  const int ops[1] = {0};
  double out[1];
  if (grid_reduce<1>(v, ops, d.partials + 20 * kMaxRedBlocks, &d.sc->ticket[T_INIT], out, sh)) {
    if (threadIdx.x == 0) finish_rhs(d.sc, out[0]);
  }
}

// The right-hand side and the Jacobi diagonal in one pass over A^T (u and theta live on the
// constraint rows only): for each variable j the same entries give sum_k A_kj u_k (plain) and
// sum_k A_kj^2 thR_k (squared).
template <int G>
__device__ __forceinline__ void group_row_dot_plain_sq(const int64_t beg, const int64_t end, const int gl,
                                                       const int32_t* __restrict__ idx, const double* __restrict__ val,
                                                       const double* __restrict__ xp, const double* __restrict__ xs,
                                                       double& op, double& os) {
  double a = 0.0, b = 0.0, a1 = 0.0, b1 = 0.0;
  int64_t e = beg + gl;
  for (; e + G < end; e += 2 * G) {
    const double v0 = __ldg(val + e), v1 = __ldg(val + e + G);
    const int i0 = __ldg(idx + e), i1 = __ldg(idx + e + G);
    a = fma(v0, __ldg(xp + i0), a);
    b = fma(v0 * v0, __ldg(xs + i0), b);
    a1 = fma(v1, __ldg(xp + i1), a1);
    b1 = fma(v1 * v1, __ldg(xs + i1), b1);
  }
  if (e < end) {
    const double v0 = __ldg(val + e);
    const int i0 = __ldg(idx + e);
    a = fma(v0, __ldg(xp + i0), a);
    b = fma(v0 * v0, __ldg(xs + i0), b);
  }
  a += a1;
  b += b1;
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  op = a;
  os = b;
}

template <int G>
__global__ void __launch_bounds__(256, 4) k_rhs_jacobi(Dev d) {
  __shared__ double sh[32];
  const double mu = d.sc->mu;
  double r2 = 0.0;
  FOR_GROUP_ROWS(G, j, ok, d.n) {
    const int64_t beg = ok ? d.AT_ptr[j] : 0, end = ok ? d.AT_ptr[j + 1] : 0;
    double atu, dth;
    group_row_dot_plain_sq<G>(beg, end, glane<G>(), d.AT_idx, d.AT_val, d.vR2, d.thR, atu, dth);
    if (ok && glane<G>() == 0) {
      d.Minv[j] = 1.0 / (d.M0[j] + dth);
      double gj = -d.rd[j] - atu;
      const double xj = d.x[j];
      if (d.fl[j]) { const double tl = xj - d.l[j]; gj -= (tl * d.zl[j] - mu) / tl; }
      if (d.fu[j]) { const double tu = d.u[j] - xj; gj += (tu * d.zu[j] - mu) / tu; }
      d.rhs[j] = gj;
      d.r[j] = gj;
      d.dx[j] = 0.0;
      r2 = fma(gj, gj, r2);
    }
  }
  if (d.aug)   // the bottom block's right-hand side (written by k_rhs_m)
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.m; k += (int64_t)gridDim.x * blockDim.x)
      r2 = fma(d.rhs[d.n + k], d.rhs[d.n + k], r2);
  double v[1] = {r2};
  const int ops[1] = {0};
  double out[1];
  if (grid_reduce<1>(v, ops, d.partials + 20 * kMaxRedBlocks, &d.sc->ticket[T_INIT], out, sh)) {
    if (threadIdx.x == 0) finish_rhs(d.sc, out[0]);
  }
}

cudaError_t launch_rhs(const Dev& d, const Geo& g, int precond, cudaStream_t st) {
  if (d.nR) cudaMemsetAsync(d.vR2, 0, sizeof(double) * d.nR, st);
  if (d.m) k_rhs_m<<<g.eM, kBlock, 0, st>>>(d);
  if (precond == PC_DENSE) {
    DISPATCH_G(d.g_at, k_rhs_n<G><<<g.gN, kBlock, 0, st>>>(d));
  } else {
    DISPATCH_G(d.g_at, k_rhs_jacobi<G><<<g.gNr, kBlock, 0, st>>>(d));
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ PCG

// v = omega o (R p).  MODE 0: inside PCG (skips once converged); MODE 1: single apply;
// MODE 2: single apply when the reduced-precision PCG asks for a residual replacement.
template <int MODE, int G>
__global__ void __launch_bounds__(256, kOpRowsMinBlocks) k_op_rows(Dev d) {
  if (MODE == 0 && d.sc->cg_done) return;
  if (MODE == 2 && !d.sc->ru_do) return;
  FOR_GROUP_ROWS(G, ri, ok, d.nR) {
    // rows in windows ordered by length (rperm), so the groups of one warp run equal trips
    const int64_t r = (ok && d.rperm) ? (int64_t)d.rperm[ri] : ri;
    const int64_t beg = ok ? d.R_ptr[r] : 0, end = ok ? d.R_ptr[r + 1] : 0;
    const double t = group_row_dot_u<G, 2>(beg, end, glane<G>(), d.R_idx, d.R_val, d.p);
    if (ok && glane<G>() == 0) {
      double v = d.omega[r] * t;
      if (MODE == 0 && d.aug) {
        // doubly augmented: top gets -A^T p_bottom; bottom q = B p_top + D p_bottom
        const int32_t k = d.rowk[r];
        if (k >= 0) {
          const double pb = d.p[d.n + k];
          v -= pb;
          d.q[d.n + k] = -t + pb * (d.s[k] / d.y[k]);
        }
      }
      d.vR[r] = v;
    }
  }
}

// v = omega o (R p) over the pieces of R's rows (FP64; one descriptor per piece of a run
// instead of one index per entry); otherwise as k_op_rows.
template <int MODE, int G>
__global__ void __launch_bounds__(256, 6) k_op_rows_runs(Dev d) {
  if (MODE == 0 && d.sc->cg_done) return;
  FOR_GROUP_ROWS(G, ri, ok, d.nR) {
    const int64_t r = (ok && d.rperm) ? (int64_t)d.rperm[ri] : ri;
    double a = 0.0;
    for_row_pieces<G>(d, r, ok, glane<G>(), [&](int64_t e, int c) { a = fma(__ldg(d.R_val + e), __ldg(d.p + c), a); });
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    const double t = a;
    if (ok && glane<G>() == 0) {
      double v = d.omega[r] * t;
      if (MODE == 0 && d.aug) {
        const int32_t k = d.rowk[r];
        if (k >= 0) {
          const double pb = d.p[d.n + k];
          v -= pb;
          d.q[d.n + k] = -t + pb * (d.s[k] / d.y[k]);
        }
      }
      d.vR[r] = v;
    }
  }
}

cudaError_t launch_op_rows_runs(const Dev& d, const Geo& g, int mode, cudaStream_t st) {
  if (!d.nR) return cudaSuccess;
  if (mode == 0) DISPATCH_G(d.g_rows, k_op_rows_runs<0, G><<<g.gRc, kBlock, 0, st>>>(d));
  else DISPATCH_G(d.g_rows, k_op_rows_runs<1, G><<<g.gRc, kBlock, 0, st>>>(d));
  return cudaGetLastError();
}

// q = R^T v + Hs p + (h0 + sigma) o p; p^T q -> alpha = rz / p^T q (last block).
// MODE 0: inside PCG; MODE 1: a single operator apply (no scalars touched); MODE 2: as 1,
// when the reduced-precision PCG asks for a residual replacement.
template <int MODE, int G>
__global__ void __launch_bounds__(256, kOpColsMinBlocks) k_op_cols(Dev d) {
  __shared__ double sh[32];
  if (MODE == 0 && d.sc->cg_done) return;
  if (MODE == 2 && !d.sc->ru_do) return;
  double pq = 0.0;
  FOR_GROUP_ROWS(G, j, ok, d.n) {
    const int64_t beg = ok ? d.RT_ptr[j] : 0, end = ok ? d.RT_ptr[j + 1] : 0;
    double acc = group_row_dot<G, false>(beg, end, glane<G>(), d.RT_idx, d.RT_val, d.vR);
    if (d.Hs_ptr) {
      const int64_t hb = ok ? d.Hs_ptr[j] : 0, he = ok ? d.Hs_ptr[j + 1] : 0;
      acc += group_row_dot<G, false>(hb, he, glane<G>(), d.Hs_idx, d.Hs_val, d.p);
    }
    if (d.ucols) acc += lr_row<G>(d, j, ok, glane<G>());
    if (ok && glane<G>() == 0) {
      const double pj = d.p[j];
      const double qj = acc + (d.h0[j] + d.sigma[j]) * pj;
      d.q[j] = qj;
      pq = fma(pj, qj, pq);
    }
  }
  if (MODE != 0) return;
  if (d.aug)   // p^T q over the bottom block too (q's bottom written by the rows pass)
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.m; k += (int64_t)gridDim.x * blockDim.x)
      pq = fma(d.p[d.n + k], d.q[d.n + k], pq);
  double v[1] = {pq};
  const int ops[1] = {0};
  double out[1];
  if (grid_reduce<1>(v, ops, d.partials + 16 * kMaxRedBlocks, &d.sc->ticket[T_PQ], out, sh)) {
    if (threadIdx.x == 0) {
      Scal* sc = d.sc;
      const double pqv = out[0];
      if (!(pqv > 0.0) || !isfinite(pqv)) {
        sc->cg_done = 1;                       // breakdown: keep the last iterate
        if (!isfinite(pqv)) sc->status = DS_NUMERICAL;
        sc->alpha = 0.0;
      } else {
        sc->alpha = sc->rz / pqv;
      }
      sc->pq = pqv;
    }
  }
}

// dx += alpha p; r -= alpha q; ||r||^2 -> convergence test.
// ZM 0 (Jacobi): z = r / M, r^T z, beta.  ZM 1 (Jacobi + low rank): z0 = r / M only.
// ZM 2 (dense): z is left to the dense apply.
template <int ZM>
__global__ void k_cg_update(Dev d) {
  __shared__ double sh[32];
  if (d.sc->cg_done) return;
  const double alpha = d.sc->alpha;
  double rr = 0.0, rz = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.nsys; j += (int64_t)gridDim.x * blockDim.x) {
    d.dx[j] = fma(alpha, d.p[j], d.dx[j]);
    const double rj = fma(-alpha, d.q[j], d.r[j]);
    d.r[j] = rj;
    rr = fma(rj, rj, rr);
    if (ZM < 2) {
      const double zj = rj * d.Minv[j];
      d.z[j] = zj;
      rz = fma(rj, zj, rz);
    }
  }
  double v[2] = {rr, rz};
  const int ops[2] = {0, 0};
  double out[2];
  if (grid_reduce<2>(v, ops, d.partials + 17 * kMaxRedBlocks, &d.sc->ticket[T_UPD], out, sh)) {
    if (threadIdx.x == 0) {
      Scal* sc = d.sc;
      sc->cg_iter += 1;
      sc->rr = out[0];
      if (!isfinite(out[0])) {
        sc->cg_done = 1;
        sc->status = DS_NUMERICAL;
      } else if (out[0] <= sc->tol2) {
        sc->cg_done = 1;
        sc->cg_conv = 1;
      } else if (sc->cg_iter >= sc->cg_max) {
        sc->cg_done = 1;
      }
      if (ZM == 0 && !sc->cg_done) {
        sc->beta = out[1] / sc->rz;
        sc->rz = out[1];
      }
    }
  }
}

// Low-rank correction (Woodbury): with z0 = M^{-1} r already in z,
//   z = z0 - M^{-1} A_s^T G^{-1} A_s z0.
// k_stiff_u: u_a = A_s z0 (one warp per stiff row).
__global__ void k_stiff_u(Dev d, int init) {
  if (!init && d.sc->cg_done) return;
  const int ns = d.sc->n_stiff;
  for (int a = gwarp(); a < ns; a += nwarps()) {
    const int32_t row = d.arow[d.stiff_k[a]];
    double u = warp_row_dot<false>(d.R_ptr[row], d.R_ptr[row + 1], d.R_idx, d.R_val, d.z);
    if ((threadIdx.x & 31) == 0) d.us[a] = u;
  }
}

// t = G^{-1} u (dense symmetric matvec, one warp per output).
__global__ void k_stiff_t(Dev d, int init) {
  if (!init && d.sc->cg_done) return;
  const int ns = d.sc->n_stiff;
  const int cap = d.stiff_cap;
  const int lane = threadIdx.x & 31;
  for (int a = gwarp(); a < ns; a += nwarps()) {
    const double* g = d.Ginv + (int64_t)a * cap;
    double acc = 0.0;
    for (int b = lane; b < ns; b += 32) acc = fma(g[b], d.us[b], acc);
    acc = warp_sum(acc);
    if (lane == 0) d.ts[a] = acc;
  }
}

// z_j = z0_j - Minv_j sum_{(a, v) in column j} v t_a; r^T z -> beta (loop) or rz (init);
// in init mode also p = z.
__global__ void k_stiff_corr(Dev d, int init) {
  __shared__ double sh[32];
  if (!init && d.sc->cg_done) return;
  const int ns = d.sc->n_stiff;
  double rz = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    double zj = d.z[j];
    if (ns > 0) {
      double acc = 0.0;
      for (int64_t t = d.sc_ptr[j]; t < d.sc_ptr[j + 1]; ++t) acc = fma(d.sc_val[t], d.ts[d.sc_slot[t]], acc);
      zj -= d.Minv[j] * acc;
      d.z[j] = zj;
    }
    if (init) {
      d.p[j] = zj;
      if (d.p32) d.p32[j] = (float)zj;
      if (d.p_df) d.p_df[j] = df_split(zj);
    }
    rz = fma(d.r[j], zj, rz);
  }
  double v[1] = {rz};
  const int ops[1] = {0};
  double out[1];
  if (grid_reduce<1>(v, ops, d.partials + 19 * kMaxRedBlocks, &d.sc->ticket[T_CORR], out, sh)) {
    if (threadIdx.x == 0) {
      Scal* sc = d.sc;
      if (init) {
        sc->rz = out[0];
      } else {
        sc->beta = out[0] / sc->rz;
        sc->rz = out[0];
      }
    }
  }
}

// Dense preconditioner apply by triangular solves in double-float pairs: z = K^{-1} r with
// s K = L L^T (the scaled K factored in pairs: L in the lower triangle of Kd, L^T mirrored
// into the upper triangle, both row-major), forward L y = r' then backward L^T z' = y, where
// r' = 2^-e r (2^e >= max |r|, exact) and z = s 2^e z'.  In blocks of 32 rows: the block's
// 32 values come from the inverse of its diagonal tile (one warp per row, a shuffle-tree sum
// of pairs: no row-by-row chain), then all threads update the remaining rows with the block's
// 32 columns while the next tile's inverse is staged in shared memory.  Thread r reads its
// row's 32 factor entries (256 contiguous bytes: after the first miss the rest hit L1).  One block of 1024
// threads; y in shared memory (n <= 2048).  r^T z -> rz / beta; init: p = z.  (PCG with the
// factor converges in one or two iterations, so this replaces forming K^{-1} once per IPM
// iteration.)
__global__ void __launch_bounds__(1024) k_dense_trsv(Dev d, int init) {
  extern __shared__ float2 y[];
  __shared__ double sh[32];
  __shared__ float2 Li[2][32][33];
  __shared__ float2 yk[32];
  if (!init && d.sc->cg_done) return;
  const int n = (int)d.n;
  const int nt = (n + 31) / 32;
  const float2* K = d.Kd;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double rmax = 0.0;
  for (int i = tid; i < n; i += blockDim.x) rmax = fmax(rmax, fabs(d.r[i]));
  rmax = block_reduce<1>(rmax, sh);
  int er = 0;
  if (rmax > 0.0 && isfinite(rmax)) frexp(rmax, &er);
  const double rs = ldexp(1.0, -er);
  for (int i = tid; i < n; i += blockDim.x) y[i] = df_split(d.r[i] * rs);
  if (nt > 0) Li[0][warp][lane] = d.chol_tinv[warp * 32 + lane];
  __syncthreads();
  // forward: L y = r'
  for (int t = 0; t < nt; ++t) {
    const int kb = t * 32, bs = min(32, n - kb), cur = t & 1;
    float h = 0.f, l = 0.f;
    if (lane < bs) df_mac(Li[cur][warp][lane], y[kb + lane], h, l);
    df_group_pair<32>(h, l);
    if (lane == 0) yk[warp] = df_fast_sum(h, l);
    __syncthreads();
    if (t + 1 < nt) Li[cur ^ 1][warp][lane] = d.chol_tinv[(int64_t)(t + 1) * 1024 + warp * 32 + lane];
    if (tid < bs) y[kb + tid] = yk[tid];
    for (int r = kb + bs + tid; r < n; r += blockDim.x) {
      const float2* Lr = K + (int64_t)r * n + kb;
      float ah = 0.f, al = 0.f;
      for (int c = 0; c < bs; ++c) df_mac(Lr[c], yk[c], ah, al);
      y[r] = df_sub_sum(y[r], ah, al);
    }
    __syncthreads();
  }
  // backward: L^T z' = y, with L^T row i in the upper triangle of row i; tile nt - 1's
  // inverse is still staged
  for (int t = nt - 1; t >= 0; --t) {
    const int kb = t * 32, bs = min(32, n - kb), cur = t & 1;
    float h = 0.f, l = 0.f;
    if (lane < bs) df_mac(Li[cur][lane][warp], y[kb + lane], h, l);
    df_group_pair<32>(h, l);
    if (lane == 0) yk[warp] = df_fast_sum(h, l);
    __syncthreads();
    if (t > 0) Li[cur ^ 1][warp][lane] = d.chol_tinv[(int64_t)(t - 1) * 1024 + warp * 32 + lane];
    if (tid < bs) y[kb + tid] = yk[tid];
    for (int r = tid; r < kb; r += blockDim.x) {
      const float2* Ur = K + (int64_t)r * n + kb;
      float ah = 0.f, al = 0.f;
      for (int c = 0; c < bs; ++c) df_mac(Ur[c], yk[c], ah, al);
      y[r] = df_sub_sum(y[r], ah, al);
    }
    __syncthreads();
  }
  const double zs = d.dense_aux[2] * ldexp(1.0, er);
  double rz = 0.0;
  for (int j = tid; j < n; j += blockDim.x) {
    const double zj = df_value(y[j].x, y[j].y) * zs;
    d.z[j] = zj;
    if (init) {
      d.p[j] = zj;
      if (d.p32) d.p32[j] = (float)zj;
      if (d.p_df) d.p_df[j] = df_split(zj);
    }
    rz = fma(d.r[j], zj, rz);
  }
  rz = block_reduce<0>(rz, sh);
  if (tid == 0) {
    Scal* sc = d.sc;
    if (init) {
      sc->rz = rz;
    } else {
      sc->beta = rz / sc->rz;
      sc->rz = rz;
    }
  }
}

// Jacobi start: z = r / M, p = z, rz = r^T z.
__global__ void k_cg_init_diag(Dev d) {
  __shared__ double sh[32];
  double rz = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.nsys; j += (int64_t)gridDim.x * blockDim.x) {
    const double zj = d.r[j] * d.Minv[j];
    d.z[j] = zj;
    d.p[j] = zj;
    if (d.p_df && j < d.n) d.p_df[j] = df_split(zj);
    rz = fma(d.r[j], zj, rz);
  }
  double v[1] = {rz};
  const int ops[1] = {0};
  double out[1];
  if (grid_reduce<1>(v, ops, d.partials + 21 * kMaxRedBlocks, &d.sc->ticket[T_CORR], out, sh)) {
    if (threadIdx.x == 0) d.sc->rz = out[0];
  }
}

// p = z + beta p; also sets the while-loop condition of the captured PCG graph.
__global__ void k_cg_p(Dev d, cudaGraphConditionalHandle h, int set_cond) {
  const int done = d.sc->cg_done;
  if (set_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, done ? 0u : 1u);
  if (done) return;
  const double beta = d.sc->beta;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.nsys; j += (int64_t)gridDim.x * blockDim.x)
  {
    const double pj = fma(beta, d.p[j], d.z[j]);
    d.p[j] = pj;
    if (d.p32) d.p32[j] = (float)pj;
    if (d.p_df && j < d.n) d.p_df[j] = df_split(pj);
  }
}

cudaError_t launch_cg_init(const Dev& d, const Geo& g, int precond, cudaStream_t st) {
  if (precond == PC_BLOCK32) return launch_block_apply(d, 1, st);
  if (precond == PC_DENSE) {
    k_dense_trsv<<<1, 1024, sizeof(float2) * d.n, st>>>(d, 1);
  } else if (precond == PC_JACOBI_LR) {
    k_cg_init_diag<<<g.eN, kBlock, 0, st>>>(d);
    const int gs = (d.stiff_cap + 7) / 8;
    k_stiff_u<<<gs, kBlock, 0, st>>>(d, 1);
    k_stiff_t<<<gs, kBlock, 0, st>>>(d, 1);
    k_stiff_corr<<<g.eN, kBlock, 0, st>>>(d, 1);
  } else {
    k_cg_init_diag<<<g.eN, kBlock, 0, st>>>(d);
  }
  return cudaGetLastError();
}

cudaError_t launch_cg_body(const Dev& d, const Geo& g, int precond, cudaGraphConditionalHandle h, cudaStream_t st,
                           bool in_graph, bool lowp) {
  if (lowp) {
    cudaError_t e = launch_op_lp(d, g, st);
    if (e != cudaSuccess) return e;
  } else if (d.mx) {
    launch_op_rows_mx(d, g, 0, st);
    launch_lr(d, d.p, 0, st);
    launch_op_cols_mx(d, g, 0, st);
  } else if (d.df) {
    launch_op_rows_df(d, g, 0, st);
    launch_lr(d, d.p, 0, st);
    launch_op_cols_df(d, g, 0, st);
  } else {
    if (d.runs) launch_op_rows_runs(d, g, 0, st);
    else if (d.nR) DISPATCH_G(d.g_rows, k_op_rows<0, G><<<g.gR64, kBlock, 0, st>>>(d));
    launch_lr(d, d.p, 0, st);
    DISPATCH_G(d.g_cols, k_op_cols<0, G><<<g.gN64, kBlock, 0, st>>>(d));
  }
  if (precond == PC_BLOCK32) {
    k_cg_update<2><<<g.eN, kBlock, 0, st>>>(d);
    launch_block_apply(d, 0, st);
  } else if (precond == PC_DENSE) {
    k_cg_update<2><<<g.eN, kBlock, 0, st>>>(d);
    k_dense_trsv<<<1, 1024, sizeof(float2) * d.n, st>>>(d, 0);
  } else if (precond == PC_JACOBI_LR) {
    k_cg_update<1><<<g.eN, kBlock, 0, st>>>(d);
    const int gs = (d.stiff_cap + 7) / 8;
    k_stiff_u<<<gs, kBlock, 0, st>>>(d, 0);
    k_stiff_t<<<gs, kBlock, 0, st>>>(d, 0);
    k_stiff_corr<<<g.eN, kBlock, 0, st>>>(d, 0);
  } else {
    k_cg_update<0><<<g.eN, kBlock, 0, st>>>(d);
  }
  k_cg_p<<<g.eN, kBlock, 0, st>>>(d, h, in_graph ? 1 : 0);
  return cudaGetLastError();
}

// The rows and the column pass of the handle's FP64-storage PCG operator alone (measurement,
// autotuning); the double-float passes read p_df, which the caller keeps current.
// The low-rank correction of the preconditioner after z0 = r / M (loop form) and the next
// search direction (with the loop condition), for the replacement PCG of lowp.cu.
cudaError_t launch_stiff_apply(const Dev& d, const Geo& g, cudaStream_t st) {
  const int gs = (d.stiff_cap + 7) / 8;
  k_stiff_u<<<gs, kBlock, 0, st>>>(d, 0);
  k_stiff_t<<<gs, kBlock, 0, st>>>(d, 0);
  k_stiff_corr<<<g.eN, kBlock, 0, st>>>(d, 0);
  return cudaGetLastError();
}

cudaError_t launch_cg_p(const Dev& d, const Geo& g, cudaGraphConditionalHandle h, bool in_graph, cudaStream_t st) {
  k_cg_p<<<g.eN, kBlock, 0, st>>>(d, h, in_graph ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_op_rows_only(const Dev& d, const Geo& g, cudaStream_t st) {
  if (d.mx) return launch_op_rows_mx(d, g, 1, st);
  if (d.df) return launch_op_rows_df(d, g, 1, st);
  if (d.runs) return launch_op_rows_runs(d, g, 1, st);
  if (d.nR) DISPATCH_G(d.g_rows, k_op_rows<1, G><<<g.gR64, kBlock, 0, st>>>(d));
  return cudaGetLastError();
}

cudaError_t launch_op_cols_only(const Dev& d, const Geo& g, cudaStream_t st) {
  // (the low-rank term uses us from the last launch_lr; the measurement does not re-run it)
  if (d.mx) return launch_op_cols_mx(d, g, 1, st);
  if (d.df) return launch_op_cols_df(d, g, 1, st);
  DISPATCH_G(d.g_cols, k_op_cols<1, G><<<g.gN64, kBlock, 0, st>>>(d));
  return cudaGetLastError();
}

// q = K p, one apply of the handle's FP64-storage PCG operator (FP64 or double-float).
cudaError_t launch_apply(const Dev& d, const Geo& g, cudaStream_t st) {
  if (d.mx) {
    launch_mirror_df(d, g, st);
    launch_op_rows_mx(d, g, 1, st);
    launch_lr(d, d.p, 0, st);
    launch_op_cols_mx(d, g, 1, st);
    return cudaGetLastError();
  }
  if (d.df) {
    launch_mirror_df(d, g, st);
    launch_op_rows_df(d, g, 1, st);
    launch_lr(d, d.p, 0, st);
    launch_op_cols_df(d, g, 1, st);
    return cudaGetLastError();
  }
  // (a reduced-storage handle keeps runs for its narrow rows pass; its FP64 applies read CSR,
  // the faster FP64 form)
  if (d.runs && d.storage == ST_F64) launch_op_rows_runs(d, g, 1, st);
  else if (d.nR) DISPATCH_G(d.g_rows, k_op_rows<1, G><<<g.gR64, kBlock, 0, st>>>(d));
  launch_lr(d, d.p, 0, st);
  DISPATCH_G(d.g_cols, k_op_cols<1, G><<<g.gN64, kBlock, 0, st>>>(d));
  return cudaGetLastError();
}

// q = K dx when the reduced-precision PCG asks for a residual replacement (ru_do), else
// nothing: the FP64 operator over the accumulated step (a copy of the bundle with p -> dx).
cudaError_t launch_apply_ru(const Dev& d, const Geo& g, cudaStream_t st) {
  Dev d2 = d;
  d2.p = d.dx;
  if (d.nR) DISPATCH_G(d.g_rows, k_op_rows<2, G><<<g.gR64, kBlock, 0, st>>>(d2));
  if (d.ucols) launch_lr(d2, d2.p, 0, st);
  DISPATCH_G(d.g_cols, k_op_cols<2, G><<<g.gN64, kBlock, 0, st>>>(d2));
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ recovery

// A dx on the constraint rows; ds = -r_p - A dx; dy = theta (A dx + r_p) - r_s / s.
template <int G>
__global__ void k_recover_m(Dev d) {
  const double mu = d.sc->mu;
  FOR_GROUP_ROWS(G, k, ok, d.m) {
    const int32_t row = ok ? d.arow[k] : 0;
    const int64_t beg = ok ? d.R_ptr[row] : 0, end = ok ? d.R_ptr[row + 1] : 0;
    const double adx = group_row_dot<G, false>(beg, end, glane<G>(), d.R_idx, d.R_val, d.dx);
    if (ok && glane<G>() == 0) {
      const double s = d.s[k];
      const double rs = s * d.y[k] - mu;
      d.ds[k] = -d.rp[k] - adx;
      // doubly augmented: dy is the solved bottom block
      d.dy[k] = d.aug ? d.dx[d.n + k] : d.theta[k] * (adx + d.rp[k]) - rs / s;
    }
  }
}

// dz_l = (-r_l - z_l dx) / t_l, dz_u = (-r_u + z_u dx) / t_u.
__global__ void k_recover_n(Dev d) {
  const double mu = d.sc->mu;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    const double xj = d.x[j], dxj = d.dx[j];
    double dzl = 0.0, dzu = 0.0;
    if (d.fl[j]) { const double tl = xj - d.l[j]; const double rl = tl * d.zl[j] - mu; dzl = (-rl - d.zl[j] * dxj) / tl; }
    if (d.fu[j]) { const double tu = d.u[j] - xj; const double ru = tu * d.zu[j] - mu; dzu = (-ru + d.zu[j] * dxj) / tu; }
    d.dzl[j] = dzl;
    d.dzu[j] = dzu;
  }
}

cudaError_t launch_recover(const Dev& d, const Geo& g, cudaStream_t st) {
  if (d.m) DISPATCH_G(d.g_rows, k_recover_m<G><<<g.gM, kBlock, 0, st>>>(d));
  k_recover_n<<<g.eN, kBlock, 0, st>>>(d);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ ratio test

static __device__ __forceinline__ double ratio_of(double v, double dv) { return dv < 0.0 ? -v / dv : INFINITY; }

__global__ void k_ratio_m(Dev d, double* part) {
  __shared__ double sh[32];
  double ap = INFINITY, ad = INFINITY;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.m; k += (int64_t)gridDim.x * blockDim.x) {
    ap = fmin(ap, ratio_of(d.s[k], d.ds[k]));
    ad = fmin(ad, ratio_of(d.y[k], d.dy[k]));
  }
  double v = block_reduce<2>(ap, sh);
  if (threadIdx.x == 0) part[0 * kMaxRedBlocks + blockIdx.x] = v;
  v = block_reduce<2>(ad, sh);
  if (threadIdx.x == 0) part[1 * kMaxRedBlocks + blockIdx.x] = v;
}

__global__ void k_ratio_n(Dev d, double* part) {
  __shared__ double sh[32];
  double ap = INFINITY, ad = INFINITY;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    const double xj = d.x[j], dxj = d.dx[j];
    if (d.fl[j]) { ap = fmin(ap, ratio_of(xj - d.l[j], dxj)); ad = fmin(ad, ratio_of(d.zl[j], d.dzl[j])); }
    if (d.fu[j]) { ap = fmin(ap, ratio_of(d.u[j] - xj, -dxj)); ad = fmin(ad, ratio_of(d.zu[j], d.dzu[j])); }
  }
  double v = block_reduce<2>(ap, sh);
  if (threadIdx.x == 0) part[2 * kMaxRedBlocks + blockIdx.x] = v;
  v = block_reduce<2>(ad, sh);
  if (threadIdx.x == 0) part[3 * kMaxRedBlocks + blockIdx.x] = v;
}

__global__ void k_ratio_final(Dev d, int gM, int gN, const double* part) {
  __shared__ double sh[32];
  auto mn = [&](int q, int nb) -> double {
    double acc = INFINITY;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc = fmin(acc, part[q * kMaxRedBlocks + b]);
    return block_reduce<2>(acc, sh);
  };
  const double ap = fmin(mn(0, gM), mn(2, gN));
  const double ad = fmin(mn(1, gM), mn(3, gN));
  if (threadIdx.x == 0) {
    Scal* sc = d.sc;
    double a_p = fmin(1.0, sc->tau * ap);
    double a_d = fmin(1.0, sc->tau * ad);
    if (sc->equal_steps) a_p = a_d = fmin(a_p, a_d);
    sc->alpha_p = a_p;
    sc->alpha_d = a_d;
  }
}

cudaError_t launch_ratio(const Dev& d, const Geo& g, cudaStream_t st) {
  double* part = d.partials + 22 * kMaxRedBlocks;
  if (d.m) k_ratio_m<<<g.eM, kBlock, 0, st>>>(d, part);
  k_ratio_n<<<g.eN, kBlock, 0, st>>>(d, part);
  k_ratio_final<<<1, 256, 0, st>>>(d, d.m ? g.eM : 0, g.eN, part);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ update

__global__ void k_update_n(Dev d) {
  const double ap = d.sc->alpha_p, ad = d.sc->alpha_d;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    d.x[j] = fma(ap, d.dx[j], d.x[j]);
    if (d.fl[j]) d.zl[j] = fma(ad, d.dzl[j], d.zl[j]);
    if (d.fu[j]) d.zu[j] = fma(ad, d.dzu[j], d.zu[j]);
  }
}

__global__ void k_update_m(Dev d) {
  const double ap = d.sc->alpha_p, ad = d.sc->alpha_d;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.m; k += (int64_t)gridDim.x * blockDim.x) {
    d.s[k] = fma(ap, d.ds[k], d.s[k]);
    d.y[k] = fma(ad, d.dy[k], d.y[k]);
  }
}

cudaError_t launch_update(const Dev& d, const Geo& g, cudaStream_t st) {
  k_update_n<<<g.eN, kBlock, 0, st>>>(d);
  if (d.m) k_update_m<<<g.eM, kBlock, 0, st>>>(d);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ precond build

cudaError_t launch_dense_build(const Dev& d, cudaStream_t st);       // dense.cu
cudaError_t launch_stiff_factor(const Dev& d, cudaStream_t st);      // dense.cu

// Before the right-hand side: stiff-row selection (JACOBI_LR).
cudaError_t launch_precond_build(const Dev& d, const Geo& g, int precond, cudaStream_t st) {
  if (precond == PC_JACOBI_LR && d.m) {
    DISPATCH_G(d.g_rows, k_stiff_ratio<G><<<g.gM, kBlock, 0, st>>>(d));
    k_stiff_compact<<<1, 1024, 0, st>>>(d);
  }
  return cudaGetLastError();
}

// After the right-hand side (which also wrote the Jacobi diagonal): the low-rank factor
// (JACOBI_LR) or the dense factor (DENSE).
cudaError_t launch_precond_finish(const Dev& d, const Geo& g, int precond, cudaStream_t st) {
  if (precond == PC_DENSE) return launch_dense_build(d, st);
  if (precond == PC_BLOCK32) return launch_block_factor(d, st);
  if (precond == PC_JACOBI_LR && d.m) {
    k_sc_count<<<g.gN, kBlock, 0, st>>>(d);
    k_sc_scan<<<1, 1024, 0, st>>>(d);
    k_sc_fill<<<g.gN, kBlock, 0, st>>>(d);
    const size_t smem = sizeof(double) * (size_t)d.stiff_cap;
    k_gram_G<<<d.stiff_cap, 256, smem, st>>>(d);
    cudaError_t e = launch_stiff_factor(d, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace ipmk
