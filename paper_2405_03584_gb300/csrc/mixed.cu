// PCG operator passes with their products split between the float64 and the float32 pipes.
//
// On GB300 the float64 pipe takes 16 SM cycles per warp multiply-add, so the FP64 passes are
// bound by it; the double-float passes (df.cu) move every product to the float32 pipe but
// then issue about 40 instructions per entry and are bound by instruction issue and latency.
// Here each trip of a lane takes B entries: the first NF on the float64 pipe (values from the
// FP64 copy, the vector's FP64 copy), the others in double-float (values from the (hi, lo)
// copy, the vector's pair copy), so both pipes work at once and each entry is still read once
// (8 bytes either way).  The two partial sums are added in float64 by one lane per row; every
// order is fixed, so results are bitwise reproducible.  Options: ipm_options.op_arith =
// IPM_ARITH_MIXED (F64 storage).
#include "state.h"

namespace ipmk {

static __device__ __forceinline__ int gwarp_x() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
static __device__ __forceinline__ int nwarps_x() { return (gridDim.x * blockDim.x) >> 5; }

#define FOR_GROUP_ROWS_X(G, r, ok, nrows)                                                                    \
  for (int64_t r##_0 = (int64_t)gwarp_x() * (32 / G); r##_0 < (nrows); r##_0 += (int64_t)nwarps_x() * (32 / G)) \
    for (int64_t r = r##_0 + (threadIdx.x & 31) / G, r##_once = 0; r##_once == 0; r##_once = 1)               \
      for (bool ok = r < (nrows), ok##_once = true; ok##_once; ok##_once = false)

#define DISPATCH_GX(g, ...)                                  \
  switch (g) {                                               \
    case 4: { constexpr int G = 4; __VA_ARGS__; } break;     \
    case 8: { constexpr int G = 8; __VA_ARGS__; } break;     \
    case 16: { constexpr int G = 16; __VA_ARGS__; } break;   \
    default: { constexpr int G = 32; __VA_ARGS__; } break;   \
  }

constexpr int kMxB = 2;    // entries per trip of a lane
constexpr int kMxNF = 1;   // of which on the float64 pipe

// Row dot by a group of G lanes with uniform trips (entries past the row's end load as 0):
// a float64 partial a and a double-float partial (h, l), each summed over the group.
template <int G>
__device__ __forceinline__ void group_row_dot_mx(const int64_t beg, const int64_t end, const int gl,
                                                 const int32_t* __restrict__ idx, const double* __restrict__ v64,
                                                 const float2* __restrict__ vdf, const double* __restrict__ x64,
                                                 const float2* __restrict__ xdf, double& a, float& h, float& l) {
  a = 0.0;
  h = 0.f;
  l = 0.f;
  const int64_t trips = (end - beg + (int64_t)kMxB * G - 1) / ((int64_t)kMxB * G);
  int64_t e = beg + gl;
  for (int64_t t = 0; t < trips; ++t, e += (int64_t)kMxB * G) {
    int i[kMxB];
    double v[kMxNF];
    float2 w[kMxB - kMxNF];
#pragma unroll
    for (int k = 0; k < kMxB; ++k) {
      const int64_t ek = e + k * G;
      const bool in = ek < end;
      i[k] = in ? __ldg(idx + ek) : 0;
      if (k < kMxNF) v[k] = in ? __ldg(v64 + ek) : 0.0;
      else w[k - kMxNF] = in ? __ldg(vdf + ek) : make_float2(0.f, 0.f);
    }
    double xv[kMxNF];
    float2 xw[kMxB - kMxNF];
#pragma unroll
    for (int k = 0; k < kMxB; ++k) {
      if (k < kMxNF) xv[k] = __ldg(x64 + i[k]);
      else xw[k - kMxNF] = __ldg(xdf + i[k]);
    }
#pragma unroll
    for (int k = 0; k < kMxNF; ++k) a = fma(v[k], xv[k], a);
#pragma unroll
    for (int k = 0; k < kMxB - kMxNF; ++k) df_mac(w[k], xw[k], h, l);
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  df_group_pair<G>(h, l);
}

// v = omega o (R p), written as float64 (vR) and as pairs (v_df) for the column pass.
// MODE 0: inside PCG (with the doubly augmented bottom block); MODE 1: one apply.
template <int MODE, int G>
__global__ void __launch_bounds__(256, 6) k_op_rows_mx(Dev d) {
  if (MODE == 0 && d.sc->cg_done) return;
  const int gl = threadIdx.x & (G - 1);
  FOR_GROUP_ROWS_X(G, ri, ok, d.nR) {
    const int64_t r = (ok && d.rperm) ? (int64_t)d.rperm[ri] : ri;
    const int64_t beg = ok ? d.R_ptr[r] : 0, end = ok ? d.R_ptr[r + 1] : 0;
    double a;
    float h, l;
    group_row_dot_mx<G>(beg, end, gl, d.R_idx, d.R_val, d.R_df, d.p, d.p_df, a, h, l);
    if (ok && gl == 0) {
      const double t = a + df_value(h, l);
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
      d.v_df[r] = df_split(v);
    }
  }
}

// q = R^T v + Hs p + U (W t) + (h0 + sigma) o p with R^T v split between the pipes; p^T q ->
// alpha = rz / p^T q (last block), as the FP64 column pass.
template <int MODE, int G>
__global__ void __launch_bounds__(256, 6) k_op_cols_mx(Dev d) {
  __shared__ double sh[32];
  if (MODE == 0 && d.sc->cg_done) return;
  const int gl = threadIdx.x & (G - 1);
  double pq = 0.0;
  FOR_GROUP_ROWS_X(G, j, ok, d.n) {
    const int64_t beg = ok ? d.RT_ptr[j] : 0, end = ok ? d.RT_ptr[j + 1] : 0;
    double a;
    float h, l;
    group_row_dot_mx<G>(beg, end, gl, d.RT_idx, d.RT_val, d.RT_df, d.vR, d.v_df, a, h, l);
    double acc = gl == 0 ? a + df_value(h, l) : 0.0;
    if (d.Hs_ptr) {
      const int64_t hb = ok ? d.Hs_ptr[j] : 0, he = ok ? d.Hs_ptr[j + 1] : 0;
      acc += group_row_dot<G, false>(hb, he, gl, d.Hs_idx, d.Hs_val, d.p);
    }
    if (d.ucols) acc += lr_row<G>(d, j, ok, gl);
    if (ok && gl == 0) {
      const double pj = d.p[j];
      const double qj = acc + (d.h0[j] + d.sigma[j]) * pj;
      d.q[j] = qj;
      pq = fma(pj, qj, pq);
    }
  }
  if (MODE == 1) return;
  if (d.aug)
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
        sc->cg_done = 1;
        if (!isfinite(pqv)) sc->status = DS_NUMERICAL;
        sc->alpha = 0.0;
      } else {
        sc->alpha = sc->rz / pqv;
      }
      sc->pq = pqv;
    }
  }
}

cudaError_t launch_op_rows_mx(const Dev& d, const Geo& g, int mode, cudaStream_t st) {
  if (!d.nR) return cudaSuccess;
  if (mode == 0) { DISPATCH_GX(d.g_rows, k_op_rows_mx<0, G><<<g.gRc, kBlock, 0, st>>>(d)); }
  else { DISPATCH_GX(d.g_rows, k_op_rows_mx<1, G><<<g.gRc, kBlock, 0, st>>>(d)); }
  return cudaGetLastError();
}

cudaError_t launch_op_cols_mx(const Dev& d, const Geo& g, int mode, cudaStream_t st) {
  if (mode == 0) { DISPATCH_GX(d.g_cols, k_op_cols_mx<0, G><<<g.gNc, kBlock, 0, st>>>(d)); }
  else { DISPATCH_GX(d.g_cols, k_op_cols_mx<1, G><<<g.gNc, kBlock, 0, st>>>(d)); }
  return cudaGetLastError();
}

}  // namespace ipmk
