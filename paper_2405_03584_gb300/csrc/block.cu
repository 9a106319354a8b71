// Block-Jacobi preconditioner over blocks of 32 consecutive variables (spot blocks):
//
//     M_b = K[J_b, J_b],   K = H + A^T Theta A + Sigma,   J_b = [32 b, 32 b + 32),
//
// the block-diagonal extension of the Jacobi diagonal the paper builds (Section 4.1.2).  K's
// blocks are split into a part fixed for the loaded QP,
//     C_b = sum_i w_R,i r_i r_i^T + Hs_bb + (U W U^T)_bb + diag(h0)     (r_i = row i of R on J_b),
// formed once (again after ipm_update_costs / ipm_set_lowrank), and the part that moves with
// the iterate, sum_k theta_k a_k a_k^T + diag(sigma) over the constraint rows, added every IPM
// iteration before each block is Cholesky-factored by one warp.  Both sums run over "segments"
// (the entries of one row that fall into one block, built at ingest and ordered by block,
// then row), in that fixed order, so the factors are bitwise reproducible.  A block whose
// factorisation meets a non-positive pivot falls back to its diagonal.
#include "state.h"

namespace ipmk {

static __device__ __forceinline__ int gwarp_b() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
static __device__ __forceinline__ int nwarps_b() { return (gridDim.x * blockDim.x) >> 5; }

// Gram of block b over its segments: thread t of 1024 owns entry (t / 32, t % 32).
// CONST 1: C_b (weights w_R, plus the H blocks and diag(h0)) into blkC.
// CONST 0: M_b = C_b + sum theta_k a_k a_k^T + diag(sigma) into blkL (factored next).
template <int CONST>
__global__ void __launch_bounds__(1024) k_block_gram(Dev d) {
  __shared__ double vec[32][33];
  __shared__ double wt[32];
  const int b = blockIdx.x;
  const int t = threadIdx.x, j = t >> 5, k = t & 31, w = t >> 5, lane = t & 31;
  const int64_t j0 = (int64_t)b * 32;
  const int64_t* sp = CONST ? d.bs_ptr : d.bc_ptr;
  const int32_t* srow = CONST ? d.bs_row : d.bc_row;
  const int64_t* sbeg = CONST ? d.bs_beg : d.bc_beg;
  const int32_t* scnt = CONST ? d.bs_cnt : d.bc_cnt;
  const int64_t s0 = sp[b], s1 = sp[b + 1];
  double acc = 0.0;
  for (int64_t sb = s0; sb < s1; sb += 32) {
    // warp w stages segment sb + w as a dense 32-vector, with its weight
    vec[w][lane] = 0.0;
    __syncwarp();
    const int64_t s = sb + w;
    if (s < s1) {
      const int32_t row = srow[s];
      const int64_t e0 = sbeg[s];
      const int cnt = scnt[s];
      if (lane < cnt) vec[w][d.R_idx[e0 + lane] - j0] = d.R_val[e0 + lane];
      if (lane == 0) wt[w] = CONST ? d.wR[row] : d.theta[d.rowk[row]];
    } else if (lane == 0) {
      wt[w] = 0.0;
    }
    __syncthreads();
    const int ns = (int)(s1 - sb < 32 ? s1 - sb : 32);
    for (int q = 0; q < ns; ++q) acc = fma(wt[q] * vec[q][j], vec[q][k], acc);
    __syncthreads();
  }
  const int64_t gj = j0 + j, gk = j0 + k;
  const bool in = gj < d.n && gk < d.n;
  if (CONST) {
    if (in) {
      if (d.Hs_ptr)   // the dense H block's entries of row gj in this block
        for (int64_t e = d.Hs_ptr[gj]; e < d.Hs_ptr[gj + 1]; ++e)
          if (d.Hs_idx[e] == gk) acc += d.Hs_val[e];
      if (d.ucols) {
        const double* uj = d.U + gj * d.ucols;
        const double* uk = d.U + gk * d.ucols;
        double a = 0.0;
        for (int64_t r = 0; r < d.ucols; ++r) a = fma(uj[r] * d.uw[r], uk[r], a);
        acc += a;
      }
      if (j == k) acc += d.h0[gj];
    }
    d.blkC[(int64_t)b * 1024 + t] = in ? acc : (j == k ? 1.0 : 0.0);
  } else {
    double m = d.blkC[(int64_t)b * 1024 + t] + acc;
    if (in && j == k) m += d.sigma[gj];
    d.blkL[(int64_t)b * 1024 + t] = in ? m : (j == k ? 1.0 : 0.0);
  }
}

// Cholesky factor of every M_b in place (lower triangle; one warp per block, lane i holds row
// i in shared memory).  A non-positive or non-finite pivot makes the block diagonal.
__global__ void __launch_bounds__(128) k_block_factor(Dev d) {
  __shared__ double a[4][32][33];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t b = gwarp_b(); b < d.nblk; b += nwarps_b()) {
    double* L = d.blkL + b * 1024;
    for (int c = 0; c < 32; ++c) a[w][lane][c] = L[lane * 32 + c];
    __syncwarp();
    const double diag0 = a[w][lane][lane];
    bool ok = true;
    for (int c = 0; c < 32; ++c) {
      const double piv = a[w][c][c];
      ok = ok && piv > 0.0 && isfinite(piv);
      const double sq = ok ? sqrt(piv) : 1.0;
      __syncwarp();
      if (lane >= c) a[w][lane][c] = lane == c ? sq : a[w][lane][c] / sq;
      __syncwarp();
      const double lc = a[w][lane][c];
      for (int q = c + 1; q <= lane; ++q) a[w][lane][q] = fma(-lc, a[w][q][c], a[w][lane][q]);
      __syncwarp();
    }
    ok = __all_sync(0xffffffffu, ok);
    for (int c = 0; c < 32; ++c)
      L[lane * 32 + c] = ok ? (c <= lane ? a[w][lane][c] : 0.0) : (c == lane ? sqrt(fmax(diag0, 1e-300)) : 0.0);
    __syncwarp();
  }
}

// z = M^{-1} r by block: forward L y = r_b, backward L^T z_b = y (one warp per block with the
// factor staged in shared memory, lane i holds y_i).  r^T z -> rz (init, also p = z) or beta
// (PCG loop), as the other preconditioners.
__global__ void __launch_bounds__(128) k_block_apply(Dev d, int init) {
  __shared__ double sh[32];
  __shared__ double a[4][32][33];
  if (!init && d.sc->cg_done) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double rz = 0.0;
  // a grid-stride loop with the same trip count in every warp of a block (the reduction below
  // needs all threads); a warp past the last block works on nothing
  const int64_t nb = d.nblk, stride = (int64_t)gridDim.x * 4;
  for (int64_t b0 = (int64_t)blockIdx.x * 4; b0 < nb; b0 += stride) {
    const int64_t b = b0 + w;
    const bool have = b < nb;
    if (have) {
      const double* L = d.blkL + b * 1024;
      for (int c = 0; c < 32; ++c) a[w][c][lane] = L[c * 32 + lane];
    }
    __syncwarp();
    const int64_t j = b * 32 + lane;
    const bool in = have && j < d.n;
    const double rj = in ? d.r[j] : 0.0;
    double y = rj;
    if (have) {
      for (int c = 0; c < 32; ++c) {
        if (lane == c) y = y / a[w][c][c];
        const double yc = __shfl_sync(0xffffffffu, y, c);
        if (lane > c) y = fma(-a[w][lane][c], yc, y);
      }
      for (int c = 31; c >= 0; --c) {
        if (lane == c) y = y / a[w][c][c];
        const double yc = __shfl_sync(0xffffffffu, y, c);
        if (lane < c) y = fma(-a[w][c][lane], yc, y);
      }
    }
    if (in) {
      d.z[j] = y;
      if (init) {
        d.p[j] = y;
        if (d.p32) d.p32[j] = (float)y;
        if (d.p_df) d.p_df[j] = df_split(y);
      }
      rz = fma(rj, y, rz);
    }
    __syncwarp();
  }
  double v[1] = {rz};
  const int ops[1] = {0};
  double out[1];
  if (grid_reduce<1>(v, ops, d.partials + 28 * kMaxRedBlocks, &d.sc->ticket[T_CORR], out, sh)) {
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

static int block_apply_grid(const Dev& d) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((d.nblk + 3) / 4, kMaxRedBlocks));
}

cudaError_t launch_block_const(const Dev& d, cudaStream_t st) {
  if (!d.nblk) return cudaSuccess;
  k_block_gram<1><<<(unsigned)d.nblk, 1024, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_block_factor(const Dev& d, cudaStream_t st) {
  k_block_gram<0><<<(unsigned)d.nblk, 1024, 0, st>>>(d);
  k_block_factor<<<block_apply_grid(d), 128, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_block_apply(const Dev& d, int init, cudaStream_t st) {
  k_block_apply<<<block_apply_grid(d), 128, 0, st>>>(d, init);
  return cudaGetLastError();
}

}  // namespace ipmk
