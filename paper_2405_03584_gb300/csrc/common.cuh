// Shared device-side definitions of the sm_103a interior point library.
//
// Layout in HBM (all float64 unless stated; one arena per handle, see api.cu):
//   R    : the "row" matrix [F; A_csr] in CSR (int64 row pointers, int32 columns).  Every
//          operator product goes through it: H's factor term is R^T diag(w_R) R (w_R = f_w on
//          F rows, 0 on A rows) and the constraint block is A = R[arow].
//   RT   : R^T in CSR (rows = variables), built once at ipm_set_qp, so that R^T v is a
//          deterministic gather (Section 4.1.1 stores the constraint transposes for the same
//          reason: transpose-free SpMV).
//   Hs   : optional explicit symmetric part of H in CSR (a dense H block is stored this way).
//   Scalars of the solve live in one device struct (Scal); kernels read and write them so
//   that no scalar crosses to the host inside an IPM iteration.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ipmk {

constexpr int kWarp = 32;
constexpr int kBlock = 256;          // threads per block of the streaming kernels
#ifndef IPM_OP_ROWS_MINB
#define IPM_OP_ROWS_MINB 6
#endif
#ifndef IPM_OP_COLS_MINB
#define IPM_OP_COLS_MINB 6
#endif
// resident blocks per SM the float64 operator passes are compiled for (one wave of blocks)
constexpr int kOpRowsMinBlocks = IPM_OP_ROWS_MINB;
constexpr int kOpColsMinBlocks = IPM_OP_COLS_MINB;
constexpr int kMaxRedBlocks = 2048;  // upper bound of blocks that write reduction partials
constexpr int kHistBins = 64;        // stiff-row ratio histogram bins (two per octave)

// Device scalars of one handle.
struct Scal {
  // barrier parameter and control
  double mu, mu0, eta, tol_kkt, tau;
  double cnorm, bnorm;               // ||c||_inf, ||b||_inf (set once)
  int ipm_iter, max_ipm, status, stop;
  int equal_steps, eta_override;     // eta_override: eta was set by the caller
  double eta_factor, eta_min, eta_max, eta_used;
  // PCG
  double rz, pq, alpha, beta, rr, rhs2, tol2;
  int cg_iter, cg_done, cg_max, cg_conv;
  // preconditioner
  double stiff_gamma, stiff_thresh;
  int n_stiff, stiff_max, max_stiff_seen, chol_fail;
  // FP64 refinement of a reduced-precision Newton step
  double tol2_outer, rr_outer, refine_eta;
  double lr_quad;               // x^T U W U^T x of the last residual summary
  // primal infeasibility certificate (Farkas): with (y, z) scaled by its largest entry,
  // |A^T y - z_l + z_u|_inf and b^T y - l^T z_l + u^T z_u
  double cert_res, cert_gap, mult_inf;
  // warm start: pairs raised to at least warm_rho * mu0_cold (mu0 of the last cold start)
  double mu0_cold, warm_rho;
  int refine_it, refine_max, cg_step_total, cg_conv_outer, fallback, fallback_total;
  int cg_fail_run;                   // consecutive Newton steps whose PCG ended unconverged
  // reduced-precision PCG with residual replacement: the true residual's norm^2 at the last
  // replacement and the flag asking for the next one
  double rr_ref;
  int ru_do, ru_restart;
  // totals of one solve (device-side IPM loop)
  long long cg_total;
  int refine_total, max_cg_step, trace_rows, trace_cap;
  // step
  double alpha_p, alpha_d;
  // residual summary at the current iterate (written by k_resid_final)
  double rel_kkt, res_primal, res_dual, res_gap, pobj, dobj, rnorm_mu, comp_mean;
  double rp_inf, rd_inf, rc_inf;
  int ncomp;
  // reduction tickets (last-block pattern); each is returned to 0 by its last block
  unsigned int ticket[8];
};

enum ScalTicket { T_PQ = 0, T_UPD = 1, T_CORR = 2, T_INIT = 3, T_HIST = 4, T_STEP = 5, T_MISC = 6, T_REF = 7 };

// Storage of the matrix values used inside PCG (mirrors enum ipm_storage).
enum Storage { ST_F64 = 0, ST_F32 = 1, ST_BF16 = 2, ST_FP8 = 3 };

// Status values written by the device (mirror enum ipm_status).
enum DevStatus { DS_RUNNING = -1, DS_OK = 0, DS_MAX_ITER = 3, DS_CG_STALL = 4, DS_NUMERICAL = 5, DS_INFEASIBLE = 6,
                 DS_TIMEOUT = 7 };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide reductions in a fixed order (warp tree, then warp 0 over the warp results).
// Every thread of the block must call them; the result is valid in every thread.
template <int OP>  // 0 sum, 1 max, 2 min
__device__ __forceinline__ double block_reduce(double v, double* sh /* >= 32 doubles */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = OP == 0 ? warp_sum(v) : (OP == 1 ? warp_max(v) : warp_min(v));
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const double id = OP == 0 ? 0.0 : (OP == 1 ? -INFINITY : INFINITY);
    double t = lane < nw ? sh[lane] : id;
    t = OP == 0 ? warp_sum(t) : (OP == 1 ? warp_max(t) : warp_min(t));
    if (lane == 0) sh[0] = t;
  }
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

// Last-block-done grid reduction.  Each block stores its partial for each of NQ quantities
// at partials[q * kMaxRedBlocks + blockIdx.x]; the last block to arrive reduces them in
// block-index order and returns true (in all of its threads) with the totals in out[].
// Deterministic for a fixed grid size.  ops[q]: 0 sum, 1 max, 2 min.
template <int NQ>
__device__ bool grid_reduce(const double (&v)[NQ], const int (&ops)[NQ], double* partials,
                            unsigned int* ticket, double (&out)[NQ], double* sh) {
  double r[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    r[q] = ops[q] == 0 ? block_reduce<0>(v[q], sh) : (ops[q] == 1 ? block_reduce<1>(v[q], sh) : block_reduce<2>(v[q], sh));
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) partials[q * kMaxRedBlocks + blockIdx.x] = r[q];
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double id = ops[q] == 0 ? 0.0 : (ops[q] == 1 ? -INFINITY : INFINITY);
    double acc = id;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
      double pv = __ldcg(partials + q * kMaxRedBlocks + b);
      acc = ops[q] == 0 ? acc + pv : (ops[q] == 1 ? fmax(acc, pv) : fmin(acc, pv));
    }
    out[q] = ops[q] == 0 ? block_reduce<0>(acc, sh) : (ops[q] == 1 ? block_reduce<1>(acc, sh) : block_reduce<2>(acc, sh));
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// Dot product of one CSR row with a dense vector, computed by one warp (all lanes return the
// sum).  Lanes take entries lane, lane+32, ...; four independent accumulators keep loads in
// flight; the combination order is fixed.
template <bool SQ>
__device__ __forceinline__ double warp_row_dot(const int64_t beg, const int64_t end, const int32_t* __restrict__ idx,
                                               const double* __restrict__ val, const double* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int64_t e = beg + lane;
  for (; e + 96 < end; e += 128) {
    double v0 = __ldg(val + e), v1 = __ldg(val + e + 32), v2 = __ldg(val + e + 64), v3 = __ldg(val + e + 96);
    int i0 = __ldg(idx + e), i1 = __ldg(idx + e + 32), i2 = __ldg(idx + e + 64), i3 = __ldg(idx + e + 96);
    if (SQ) { v0 *= v0; v1 *= v1; v2 *= v2; v3 *= v3; }
    a0 = fma(v0, __ldg(x + i0), a0);
    a1 = fma(v1, __ldg(x + i1), a1);
    a2 = fma(v2, __ldg(x + i2), a2);
    a3 = fma(v3, __ldg(x + i3), a3);
  }
  for (; e < end; e += 32) {
    double v0 = __ldg(val + e);
    if (SQ) v0 *= v0;
    a0 = fma(v0, __ldg(x + __ldg(idx + e)), a0);
  }
  return warp_sum((a0 + a1) + (a2 + a3));
}

// Dot product of one CSR row with a dense vector by a group of G consecutive lanes (G divides
// 32; all lanes of the warp must call it, each with its own row).  GB300 issues a float64
// warp instruction over many cycles, so the reduction is the cost to minimise: with G lanes a
// row costs nnz/G fused multiply-adds per lane plus log2(G) + 1 adds, against 5 + 3 adds for a
// whole-warp row.  Lane gl of the group takes entries gl, gl + G, ...; two accumulators keep
// loads in flight; the combination order is fixed.
// Uniform-trip row dot: every lane of the group runs ceil(len / (B G)) trips of B entries;
// entries past the row's end load as 0 with index 0, so no lane idles in a divergent tail
// (on GB300 the float64 pipe, which issues for every lane of a warp instruction, is the limit
// of these kernels).  Short trips keep the padding of the last trip small: measured on the RT
// rows pass, B = 2 with 6 blocks per SM 135 us, the 8-entry divergent-tail form 140 us,
// B = 4 138 us, B = 8 150 us.
template <int G, int B>
__device__ __forceinline__ double group_row_dot_u(const int64_t beg, const int64_t end, const int gl,
                                                  const int32_t* __restrict__ idx, const double* __restrict__ val,
                                                  const double* __restrict__ x) {
  double a = 0.0;
  const int64_t trips = (end - beg + (int64_t)B * G - 1) / ((int64_t)B * G);
  int64_t e = beg + gl;
  for (int64_t t = 0; t < trips; ++t, e += (int64_t)B * G) {
    double v[B];
    int i[B];
    double xv[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int64_t ek = e + k * G;
      const bool in = ek < end;
      v[k] = in ? __ldg(val + ek) : 0.0;
      i[k] = in ? __ldg(idx + ek) : 0;
    }
#pragma unroll
    for (int k = 0; k < B; ++k) xv[k] = __ldg(x + i[k]);
#pragma unroll
    for (int k = 0; k < B; ++k) a = fma(v[k], xv[k], a);
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}

template <int G, bool SQ>
__device__ __forceinline__ double group_row_dot(const int64_t beg, const int64_t end, const int gl,
                                                const int32_t* __restrict__ idx, const double* __restrict__ val,
                                                const double* __restrict__ x) {
  // Eight entries per trip: all value and index loads first, then all gathers, then the
  // multiply-adds into one accumulator (the float64 pipe, not the add latency, is the limit).
  double a = 0.0;
  int64_t e = beg + gl;
  for (; e + 7 * G < end; e += 8 * G) {
    double v[8];
    int i[8];
    double xv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v[k] = __ldg(val + e + k * G);
      i[k] = __ldg(idx + e + k * G);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) xv[k] = __ldg(x + i[k]);
#pragma unroll
    for (int k = 0; k < 8; ++k) a = fma(SQ ? v[k] * v[k] : v[k], xv[k], a);
  }
  for (; e < end; e += G) {
    const double v0 = __ldg(val + e);
    a = fma(SQ ? v0 * v0 : v0, __ldg(x + __ldg(idx + e)), a);
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}

// Two vectors through the same matrix row (one pass over the row), by a group of G lanes.
template <int G>
__device__ __forceinline__ void group_row_dot2(const int64_t beg, const int64_t end, const int gl,
                                               const int32_t* __restrict__ idx, const double* __restrict__ val,
                                               const double* __restrict__ x1, const double* __restrict__ x2,
                                               double& o1, double& o2) {
  double a = 0.0, b = 0.0;
  for (int64_t e = beg + gl; e < end; e += G) {
    const double v = __ldg(val + e);
    const int i = __ldg(idx + e);
    a = fma(v, __ldg(x1 + i), a);
    b = fma(v, __ldg(x2 + i), b);
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  o1 = a;
  o2 = b;
}

// Same, over two vectors at once (one pass over the matrix).
__device__ __forceinline__ void warp_row_dot2(const int64_t beg, const int64_t end, const int32_t* __restrict__ idx,
                                              const double* __restrict__ val, const double* __restrict__ x1,
                                              const double* __restrict__ x2, double& o1, double& o2) {
  const int lane = threadIdx.x & 31;
  double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
  int64_t e = beg + lane;
  for (; e + 32 < end; e += 64) {
    double v0 = __ldg(val + e), v1 = __ldg(val + e + 32);
    int i0 = __ldg(idx + e), i1 = __ldg(idx + e + 32);
    a0 = fma(v0, __ldg(x1 + i0), a0);
    b0 = fma(v0, __ldg(x2 + i0), b0);
    a1 = fma(v1, __ldg(x1 + i1), a1);
    b1 = fma(v1, __ldg(x2 + i1), b1);
  }
  for (; e < end; e += 32) {
    double v0 = __ldg(val + e);
    int i0 = __ldg(idx + e);
    a0 = fma(v0, __ldg(x1 + i0), a0);
    b0 = fma(v0, __ldg(x2 + i0), b0);
  }
  o1 = warp_sum(a0 + a1);
  o2 = warp_sum(b0 + b1);
}

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

// ---------------------------------------------------------------- double-float arithmetic
//
// A float64 value x is carried as an unevaluated pair of float32 (hi, lo) with hi = fl32(x)
// and lo = fl32(x - hi): 48 significant bits, the same 8 bytes as the double.  Products and
// sums of such pairs are formed on the float32 pipe with error-free transformations:
// Dekker's product (the rounding error of a * b is fma(a, b, -fl(a * b)) exactly; Dekker
// 1971, with the fused multiply-add in place of his splitting) and Knuth's two-sum (s =
// fl(a + b), e = (a - (s - bb)) + (b - bb) with bb = s - a gives a + b = s + e exactly; Knuth,
// TAOCP vol. 2, 4.2.2).  The _rn intrinsics are never contracted into fused operations, which
// the transformations rely on.
__device__ __forceinline__ float2 df_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double df_value(float h, float l) { return (double)h + (double)l; }

// s + e = a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (h, l) += a * x for double-float a, x: the high product and its exact error (Dekker), the
// two cross terms into the error (the lo * lo term is below the pair's precision), the high
// product added to h by two-sum, every error term into l.
__device__ __forceinline__ void df_mac(const float2 a, const float2 x, float& h, float& l) {
  const float p = __fmul_rn(a.x, x.x);
  float e = __fmaf_rn(a.x, x.x, -p);
  e = __fmaf_rn(a.x, x.y, e);
  e = __fmaf_rn(a.y, x.x, e);
  float s, t;
  two_sum(h, p, s, t);
  h = s;
  l = __fadd_rn(l, __fadd_rn(t, e));
}

// (h, l) -> a normalised pair h' + l' = h + l (|l| small against |h|: Dekker's fast two-sum)
__device__ __forceinline__ float2 df_fast_sum(float h, float l) {
  const float s = __fadd_rn(h, l);
  return make_float2(s, __fsub_rn(l, __fsub_rn(s, h)));
}

// a - (h + l) for a normalised pair a and an accumulated pair (h, l), normalised
__device__ __forceinline__ float2 df_sub_sum(float2 a, float h, float l) {
  float s, t;
  two_sum(a.x, -h, s, t);
  t = __fadd_rn(t, __fsub_rn(a.y, l));
  return df_fast_sum(s, t);
}

// Sum of the pairs of a group of G lanes in place (fixed butterfly order; every lane of the
// group gets the total pair).
template <int G>
__device__ __forceinline__ void df_group_pair(float& h, float& l) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    float s, t;
    two_sum(h, oh, s, t);
    h = s;
    l = __fadd_rn(__fadd_rn(l, ol), t);
  }
}

// The same, returned as one float64 value.
template <int G>
__device__ __forceinline__ double df_group_sum(float h, float l) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    // both partners form the same pair: s and the exact error of h + oh do not depend on the
    // operand order, and a float32 addition is commutative
    float s, t;
    two_sum(h, oh, s, t);
    h = s;
    l = __fadd_rn(__fadd_rn(l, ol), t);
  }
  return df_value(h, l);
}

}  // namespace ipmk
