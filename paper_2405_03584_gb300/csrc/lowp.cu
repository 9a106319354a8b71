// Reduced-precision operator and FP64 iterative refinement of the Newton step.
//
// The matrix values of R and R^T are stored a second time in FP32, BF16 or FP8-E4M3 with one
// FP32 scale per row of R (R~_ij = s_i q_ij, q_ij = round(R_ij / s_i)); the int32 index arrays
// are shared with the FP64 copy.  Inside PCG the operator
//     K~ p = R~^T (omega o (R~ p)) + Hs p + (h0 + sigma) o p
// reads the narrow values and an FP32 mirror of p and accumulates in FP32 (the fast pipe);
// K~ is exactly symmetric, so CG stays valid.  The Newton step keeps FP64 accuracy by
// refinement: dx <- dx + K~^{-1}(rhs - K dx) with the residual formed by the FP64 operator,
// until ||rhs - K dx|| <= eta ||rhs||.  Residuals, the refinement residual and every reduction
// stay in FP64.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "state.h"

namespace ipmk {

static __device__ __forceinline__ int gwarp_l() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
static __device__ __forceinline__ int nwarps_l() { return (gridDim.x * blockDim.x) >> 5; }

template <int S> struct StorageT;
template <> struct StorageT<ST_F32> {
  using T = float;
  static constexpr float qmax = 1.0f;
  static __device__ __forceinline__ float dec(T v) { return v; }
  static __device__ __forceinline__ T enc(float v) { return v; }
};
template <> struct StorageT<ST_BF16> {
  using T = __nv_bfloat16;
  static constexpr float qmax = 1.0f;
  static __device__ __forceinline__ float dec(T v) { return __bfloat162float(v); }
  static __device__ __forceinline__ T enc(float v) { return __float2bfloat16_rn(v); }
};
template <> struct StorageT<ST_FP8> {
  using T = __nv_fp8_e4m3;
  static constexpr float qmax = 448.0f;
  static __device__ __forceinline__ float dec(T v) { return static_cast<float>(v); }
  static __device__ __forceinline__ T enc(float v) { return T(v); }
};

// Per-row scale s_i = max_j |R_ij| / qmax (1 for an empty or zero row).
template <int S>
__global__ void k_quant_scale(Dev d) {
  for (int64_t r = gwarp_l(); r < d.nR; r += nwarps_l()) {
    double mx = 0.0;
    for (int64_t e = d.R_ptr[r] + (threadIdx.x & 31); e < d.R_ptr[r + 1]; e += 32) mx = fmax(mx, fabs(d.R_val[e]));
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) d.scaleR[r] = mx > 0.0 ? (float)(mx / (double)StorageT<S>::qmax) : 1.0f;
  }
}

template <int S>
__global__ void k_quant_rows(Dev d) {
  using T = typename StorageT<S>::T;
  T* q = static_cast<T*>(d.Rq);
  for (int64_t r = gwarp_l(); r < d.nR; r += nwarps_l()) {
    const double s = (double)d.scaleR[r];
    for (int64_t e = d.R_ptr[r] + (threadIdx.x & 31); e < d.R_ptr[r + 1]; e += 32)
      q[e] = StorageT<S>::enc((float)(d.R_val[e] / s));
  }
}

template <int S>
__global__ void k_quant_rt(Dev d) {
  using T = typename StorageT<S>::T;
  T* q = static_cast<T*>(d.RTq);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < d.nnzR; e += (int64_t)gridDim.x * blockDim.x)
    q[e] = StorageT<S>::enc((float)(d.RT_val[e] / (double)d.scaleR[d.RT_idx[e]]));
}

cudaError_t launch_quantize(const Dev& d, cudaStream_t st) {
  if (d.storage == ST_F64 || d.nR == 0) return cudaSuccess;
  const int gb = (int)std::min<int64_t>((d.nR + 7) / 8, 4096);
  const int ge = (int)std::min<int64_t>((d.nnzR + 255) / 256, 8192);
  switch (d.storage) {
    case ST_F32: k_quant_scale<ST_F32><<<gb, 256, 0, st>>>(d); k_quant_rows<ST_F32><<<gb, 256, 0, st>>>(d); k_quant_rt<ST_F32><<<ge, 256, 0, st>>>(d); break;
    case ST_BF16: k_quant_scale<ST_BF16><<<gb, 256, 0, st>>>(d); k_quant_rows<ST_BF16><<<gb, 256, 0, st>>>(d); k_quant_rt<ST_BF16><<<ge, 256, 0, st>>>(d); break;
    default: k_quant_scale<ST_FP8><<<gb, 256, 0, st>>>(d); k_quant_rows<ST_FP8><<<gb, 256, 0, st>>>(d); k_quant_rt<ST_FP8><<<ge, 256, 0, st>>>(d); break;
  }
  return cudaGetLastError();
}

// C stored values of type T decoded to FP32 from one aligned vector load.
template <int S> struct Chunk;
template <> struct Chunk<ST_F32> {
  static constexpr int C = 4;   // elements per 16-byte load
  static __device__ __forceinline__ void load(const float* p, float* v) {
    const float4 u = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
  }
};
template <> struct Chunk<ST_BF16> {
  static constexpr int C = 8;
  static __device__ __forceinline__ void load(const __nv_bfloat16* p, float* v) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = __uint_as_float(w[k] << 16);          // bf16 = the high half of an fp32
      v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
  }
};
template <> struct Chunk<ST_FP8> {
  static constexpr int C = 8;   // 8-byte loads: as many elements per chunk as BF16
  static __device__ __forceinline__ void load(const __nv_fp8_e4m3* p, float* v) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    const unsigned w[2] = {u.x, u.y};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const __nv_fp8x2_e4m3 lo = *reinterpret_cast<const __nv_fp8x2_e4m3*>(reinterpret_cast<const unsigned short*>(&w[k]));
      const __nv_fp8x2_e4m3 hi = *reinterpret_cast<const __nv_fp8x2_e4m3*>(reinterpret_cast<const unsigned short*>(&w[k]) + 1);
      const float2 a = static_cast<float2>(lo), b = static_cast<float2>(hi);
      v[4 * k] = a.x; v[4 * k + 1] = a.y; v[4 * k + 2] = b.x; v[4 * k + 3] = b.y;
    }
  }
};

// FP32 dot of a stored row with an FP32 vector by a group of G lanes.  The row is split into
// a head up to the first chunk boundary, whole chunks of C elements (one vector load of the
// C values, 16 bytes for F32 and BF16 and 8 for FP8, and C/4 16-byte index loads per chunk;
// chunk c taken by lane c mod G, two chunks in flight per lane) and a tail; one accumulator
// per lane, then a shuffle reduction over the group.  Value and index arrays are 256-byte
// aligned, so an element offset that is a multiple of C (>= 4) aligns both loads.
template <int S, int G>
__device__ __forceinline__ float group_row_dot_lp(const int64_t beg, const int64_t end, const int gl,
                                                  const int32_t* __restrict__ idx,
                                                  const typename StorageT<S>::T* __restrict__ val,
                                                  const float* __restrict__ x) {
  constexpr int C = Chunk<S>::C;
  float a = 0.f;
  int64_t a0 = (beg + C - 1) & ~(int64_t)(C - 1);
  if (a0 > end) a0 = end;
  for (int64_t e = beg + gl; e < a0; e += G) a = fmaf(StorageT<S>::dec(val[e]), __ldg(x + __ldg(idx + e)), a);
  const int64_t nch = (end - a0) / C;
  int64_t c = gl;
  for (; c + G < nch; c += 2 * G) {
    const int64_t e0 = a0 + c * C, e1 = e0 + (int64_t)G * C;
    float v0[C], v1[C];
    int i0[C], i1[C];
    Chunk<S>::load(val + e0, v0);
    Chunk<S>::load(val + e1, v1);
#pragma unroll
    for (int k = 0; k < C / 4; ++k) {
      const int4 t0 = __ldg(reinterpret_cast<const int4*>(idx + e0) + k);
      const int4 t1 = __ldg(reinterpret_cast<const int4*>(idx + e1) + k);
      i0[4 * k] = t0.x; i0[4 * k + 1] = t0.y; i0[4 * k + 2] = t0.z; i0[4 * k + 3] = t0.w;
      i1[4 * k] = t1.x; i1[4 * k + 1] = t1.y; i1[4 * k + 2] = t1.z; i1[4 * k + 3] = t1.w;
    }
#pragma unroll
    for (int k = 0; k < C; ++k) a = fmaf(v0[k], __ldg(x + i0[k]), a);
#pragma unroll
    for (int k = 0; k < C; ++k) a = fmaf(v1[k], __ldg(x + i1[k]), a);
  }
  if (c < nch) {
    const int64_t e0 = a0 + c * C;
    float v0[C];
    int i0[C];
    Chunk<S>::load(val + e0, v0);
#pragma unroll
    for (int k = 0; k < C / 4; ++k) {
      const int4 t0 = __ldg(reinterpret_cast<const int4*>(idx + e0) + k);
      i0[4 * k] = t0.x; i0[4 * k + 1] = t0.y; i0[4 * k + 2] = t0.z; i0[4 * k + 3] = t0.w;
    }
#pragma unroll
    for (int k = 0; k < C; ++k) a = fmaf(v0[k], __ldg(x + i0[k]), a);
  }
  for (int64_t e = a0 + nch * C + gl; e < end; e += G) a = fmaf(StorageT<S>::dec(val[e]), __ldg(x + __ldg(idx + e)), a);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}

#define FOR_GROUP_ROWS_L(G, r, ok, nrows)                                                                    \
  for (int64_t r##_0 = (int64_t)gwarp_l() * (32 / G); r##_0 < (nrows); r##_0 += (int64_t)nwarps_l() * (32 / G)) \
    for (int64_t r = r##_0 + (threadIdx.x & 31) / G, r##_once = 0; r##_once == 0; r##_once = 1)               \
      for (bool ok = r < (nrows), ok##_once = true; ok##_once; ok##_once = false)

// Exact FP64 part of the operator for the stiff rows (JACOBI_LR): u_a = theta_a (A_a . p).
// Their narrow copy is left out of K~ (omega_lp = w_R + theta on moderate rows only), so the
// rows whose theta dominates are never rounded: K~ = R~^T diag(w + theta_mod) R~ + A_s^T Theta_s A_s.
__global__ void k_stiff_op_u(Dev d) {
  if (d.sc->cg_done) return;
  const int ns = d.sc->n_stiff;
  for (int a = gwarp_l(); a < ns; a += nwarps_l()) {
    const int32_t k = d.stiff_k[a];
    const int32_t row = d.arow[k];
    const double u = warp_row_dot<false>(d.R_ptr[row], d.R_ptr[row + 1], d.R_idx, d.R_val, d.p);
    if ((threadIdx.x & 31) == 0) d.us2[a] = d.theta[k] * u;
  }
}

// w_i = s_i^2 (w_R,i + thR_i) (q_i . p32)   (FP32 result; thR = theta on moderate rows).
// Rows in natural order: the length order of the FP64 rows pass made this L1-bound pass
// slower (72 -> 90 us on the RT rows, BF16), the gathers of neighbouring rows sharing lines.
template <int S, int G>
__global__ void k_op_rows_lp(Dev d, int standalone) {
  if (!standalone && d.sc->cg_done) return;
  using T = typename StorageT<S>::T;
  const T* q = static_cast<const T*>(d.Rq);
  const int gl = threadIdx.x & (G - 1);
  FOR_GROUP_ROWS_L(G, r, ok, d.nR) {
    const int64_t beg = ok ? d.R_ptr[r] : 0, end = ok ? d.R_ptr[r + 1] : 0;
    const float t = group_row_dot_lp<S, G>(beg, end, gl, d.R_idx, q, d.p32);
    if (ok && gl == 0) {
      const double s = (double)d.scaleR[r];
      d.w32[r] = (float)((d.wR[r] + d.thR[r]) * s * s * (double)t);
    }
  }
}

// ---------------------------------------------------------------- gap layout of R^T
//
// The reduced-precision column pass reads R^T's row indices as 16-bit gaps: within a column
// the rows ascend, so slot s holds g_s = row_s - row_{s-1} (the column's first row is kept in
// gp_base, its gap is 0).  A gap above 65535 is bridged by filler slots of gap 65535 and value
// 0; every column is padded with slots of gap 0 and value 0 to a whole number of 8-slot
// chunks.  Index bytes per entry: 2 instead of 4.  A lane decodes a chunk of 8 slots by a
// running sum, the group adds the lane totals by a shuffle scan, and a carry moves from one
// trip of chunks to the next.

// Slots of column j: its entries, the fillers of its wide gaps, padding to a multiple of 8.
__global__ void k_gap_count(Dev d, int32_t* __restrict__ slots) {
  const int lane = threadIdx.x & 31;
  for (int64_t j = gwarp_l(); j < d.n; j += nwarps_l()) {
    const int64_t beg = d.RT_ptr[j], end = d.RT_ptr[j + 1];
    int64_t f = 0;
    for (int64_t e = beg + 1 + lane; e < end; e += 32) f += (int64_t)(d.RT_idx[e] - d.RT_idx[e - 1] - 1) / 65535;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0) slots[j] = (int32_t)(((end - beg) + f + 7) & ~(int64_t)7);
  }
}

// Fills the gap layout of column j (one warp per column): each entry's slot is its position
// plus the fillers before it (a ballot-free prefix over the warp's 32 entries, then a carry).
template <int S>
__global__ void k_gap_fill(Dev d) {
  using T = typename StorageT<S>::T;
  const int lane = threadIdx.x & 31;
  T* q = static_cast<T*>(const_cast<void*>(d.gp_q));
  uint16_t* g = const_cast<uint16_t*>(d.gp_d);
  for (int64_t j = gwarp_l(); j < d.n; j += nwarps_l()) {
    const int64_t beg = d.RT_ptr[j], end = d.RT_ptr[j + 1];
    const int64_t s0 = d.gp_ptr[j], s1 = d.gp_ptr[j + 1];
    if (lane == 0) const_cast<int32_t*>(d.gp_base)[j] = end > beg ? d.RT_idx[beg] : 0;
    int64_t next = s0;   // first slot after the entries placed so far
    for (int64_t e0 = beg; e0 < end; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool in = e < end;
      const int64_t gap = (in && e > beg) ? (int64_t)(d.RT_idx[e] - d.RT_idx[e - 1]) : 0;
      const int64_t f = gap > 0 ? (gap - 1) / 65535 : 0;
      int64_t c = in ? f + 1 : 0;              // slots this entry takes (fillers + itself)
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, c, o);
        if (lane >= o) c += t;
      }
      const int64_t pos = next + c - 1;        // the entry's own slot
      if (in) {
        for (int64_t k = 0; k < f; ++k) {
          g[pos - f + k] = 65535;
          q[pos - f + k] = StorageT<S>::enc(0.f);
        }
        g[pos] = (uint16_t)(gap - f * 65535);
        q[pos] = StorageT<S>::enc((float)(d.RT_val[e] / (double)d.scaleR[d.RT_idx[e]]));
      }
      next += __shfl_sync(0xffffffffu, c, 31);
    }
    for (int64_t s = next + lane; s < s1; s += 32) {
      g[s] = 0;
      q[s] = StorageT<S>::enc(0.f);
    }
  }
}

// Eight consecutive stored values from one aligned load.
template <int S> struct Chunk8;
template <> struct Chunk8<ST_F32> {
  static __device__ __forceinline__ void load(const float* p, float* v) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
};
template <> struct Chunk8<ST_BF16> {
  static __device__ __forceinline__ void load(const __nv_bfloat16* p, float* v) { Chunk<ST_BF16>::load(p, v); }
};
template <> struct Chunk8<ST_FP8> {
  static __device__ __forceinline__ void load(const __nv_fp8_e4m3* p, float* v) { Chunk<ST_FP8>::load(p, v); }
};

// FP32 dot of column j (gap layout) with w32 by a group of G lanes: lane gl takes chunks
// gl, gl + G, ... (8 slots each); trip counts are uniform over the warp.
template <int S, int G>
__device__ __forceinline__ float group_gap_dot_lp(const Dev& d, const int64_t j, const bool ok, const int gl) {
  using T = typename StorageT<S>::T;
  const T* q = static_cast<const T*>(d.gp_q);
  const int64_t s0 = ok ? d.gp_ptr[j] : 0, s1 = ok ? d.gp_ptr[j + 1] : 0;
  const unsigned nch = (unsigned)((s1 - s0) >> 3);
  const unsigned trips = (__reduce_max_sync(0xffffffffu, nch) + G - 1) / G;
  int64_t carry = ok ? d.gp_base[j] : 0;     // row of the slot before the trip's first chunk
  float a = 0.f;
  for (unsigned t = 0; t < trips; ++t) {
    const unsigned c = t * G + gl;
    const bool valid = c < nch;
    const int64_t sb = s0 + 8 * (int64_t)c;
    uint4 gd = make_uint4(0, 0, 0, 0);
    float v[8];
    if (valid) {
      gd = __ldg(reinterpret_cast<const uint4*>(d.gp_d + sb));
      Chunk8<S>::load(q + sb, v);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = 0.f;
    }
    const unsigned w[4] = {gd.x, gd.y, gd.z, gd.w};
    int run[8];
    int acc = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc += (int)(w[k] & 0xffffu);
      run[2 * k] = acc;
      acc += (int)(w[k] >> 16);
      run[2 * k + 1] = acc;
    }
    // exclusive scan of the lane totals over the group (width G)
    int incl = acc;
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      const int t2 = __shfl_up_sync(0xffffffffu, incl, o, G);
      if ((gl & (G - 1)) >= o) incl += t2;
    }
    const int64_t base = carry + (incl - acc);
#pragma unroll
    for (int k = 0; k < 8; ++k) a = fmaf(v[k], __ldg(d.w32 + (base + run[k])), a);
    carry += __shfl_sync(0xffffffffu, incl, G - 1, G);
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}

// q_j = sum_i q_ij w_i + Hs p + (h0 + sigma) p;  p^T q -> alpha (last block), as k_op_cols.
// GAP: R^T read in the gap layout (16-bit row gaps) instead of CSR.
template <int S, int G, bool GAP>
__global__ void __launch_bounds__(256, 6) k_op_cols_lp(Dev d, int standalone) {
  __shared__ double sh[32];
  if (!standalone && d.sc->cg_done) return;
  using T = typename StorageT<S>::T;
  const T* q = static_cast<const T*>(d.RTq);
  const int gl = threadIdx.x & (G - 1);
  const bool stiff = d.sc->n_stiff > 0;
  double pq = 0.0;
  FOR_GROUP_ROWS_L(G, j, ok, d.n) {
    float acc;
    if (GAP) {
      acc = group_gap_dot_lp<S, G>(d, j, ok, gl);
    } else {
      const int64_t beg = ok ? d.RT_ptr[j] : 0, end = ok ? d.RT_ptr[j + 1] : 0;
      acc = group_row_dot_lp<S, G>(beg, end, gl, d.RT_idx, q, d.w32);
    }
    double hs = 0.0;
    if (d.Hs_ptr) {
      const int64_t hb = ok ? d.Hs_ptr[j] : 0, he = ok ? d.Hs_ptr[j + 1] : 0;
      hs = group_row_dot<G, false>(hb, he, gl, d.Hs_idx, d.Hs_val, d.p);
    }
    if (d.ucols) hs += lr_row<G>(d, j, ok, gl);   // low-rank term kept in FP64
    if (ok && gl == 0) {
      const double pj = d.p[j];
      double st = 0.0;
      if (stiff)
        for (int64_t t = d.sc_ptr[j]; t < d.sc_ptr[j + 1]; ++t) st = fma(d.sc_val[t], d.us2[d.sc_slot[t]], st);
      const double qj = (double)acc + hs + st + (d.h0[j] + d.sigma[j]) * pj;
      d.q[j] = qj;
      pq = fma(pj, qj, pq);
    }
  }
  if (standalone) return;
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

#define DISPATCH_SG(s, g, ...)                                                                   \
  do {                                                                                           \
    if ((s) == ST_F32) { constexpr int S = ST_F32; DISPATCH_GL(g, __VA_ARGS__); }                \
    else if ((s) == ST_BF16) { constexpr int S = ST_BF16; DISPATCH_GL(g, __VA_ARGS__); }         \
    else { constexpr int S = ST_FP8; DISPATCH_GL(g, __VA_ARGS__); }                              \
  } while (0)
#define DISPATCH_GL(g, ...)                                   \
  switch (g) {                                                \
    case 4: { constexpr int G = 4; __VA_ARGS__; } break;      \
    case 8: { constexpr int G = 8; __VA_ARGS__; } break;      \
    case 16: { constexpr int G = 16; __VA_ARGS__; } break;    \
    default: { constexpr int G = 32; __VA_ARGS__; } break;    \
  }

// The reduced-precision rows pass over the pieces of R's rows: one descriptor per piece of a
// run instead of one index per entry, the narrow values and the FP32 vector at consecutive
// addresses (otherwise as k_op_rows_lp).
template <int S, int G>
__global__ void __launch_bounds__(256, 6) k_op_rows_lp_runs(Dev d, int standalone) {
  if (!standalone && d.sc->cg_done) return;
  using T = typename StorageT<S>::T;
  const T* q = static_cast<const T*>(d.Rq);
  const int gl = threadIdx.x & (G - 1);
  FOR_GROUP_ROWS_L(G, r, ok, d.nR) {
    float a = 0.f;
    for_row_pieces<G>(d, r, ok, gl, [&](int64_t e, int c) { a = fmaf(StorageT<S>::dec(q[e]), __ldg(d.p32 + c), a); });
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (ok && gl == 0) {
      const double s = (double)d.scaleR[r];
      d.w32[r] = (float)((d.wR[r] + d.thR[r]) * s * s * (double)a);
    }
  }
}

static void launch_rows_lp(const Dev& d, const Geo& g, int standalone, cudaStream_t st) {
  if (!d.nR) return;
  if (d.ntiles) {
    launch_op_rows_staged(d, standalone ? 1 : 0, st);
    return;
  }
  if (d.runs) DISPATCH_SG(d.storage, d.g_rows, k_op_rows_lp_runs<S, G><<<g.gRc, kBlock, 0, st>>>(d, standalone));
  else DISPATCH_SG(d.storage, d.g_rows, k_op_rows_lp<S, G><<<g.gR, kBlock, 0, st>>>(d, standalone));
}

cudaError_t launch_op_rows_lp_runs(const Dev& d, const Geo& g, int standalone, cudaStream_t st) {
  if (d.nR) DISPATCH_SG(d.storage, d.g_rows, k_op_rows_lp_runs<S, G><<<g.gRc, kBlock, 0, st>>>(d, standalone));
  return cudaGetLastError();
}

cudaError_t launch_op_lp(const Dev& d, const Geo& g, cudaStream_t st) {
  k_stiff_op_u<<<(d.stiff_cap + 7) / 8, kBlock, 0, st>>>(d);
  launch_lr(d, d.p, 0, st);
  launch_rows_lp(d, g, 0, st);
  if (d.gap) DISPATCH_SG(d.storage, d.g_cols, k_op_cols_lp<S, G, true><<<g.gNc, kBlock, 0, st>>>(d, 0));
  else DISPATCH_SG(d.storage, d.g_cols, k_op_cols_lp<S, G, false><<<g.gNc, kBlock, 0, st>>>(d, 0));
  return cudaGetLastError();
}

// The two reduced-precision passes alone (measurement): no scalars read or written; p32 must
// hold the FP32 mirror of p.
cudaError_t launch_op_rows_lp_only(const Dev& d, const Geo& g, cudaStream_t st) {
  launch_rows_lp(d, g, 1, st);
  return cudaGetLastError();
}

cudaError_t launch_op_cols_lp_only(const Dev& d, const Geo& g, cudaStream_t st) {
  if (d.gap) DISPATCH_SG(d.storage, d.g_cols, k_op_cols_lp<S, G, true><<<g.gNc, kBlock, 0, st>>>(d, 1));
  else DISPATCH_SG(d.storage, d.g_cols, k_op_cols_lp<S, G, false><<<g.gNc, kBlock, 0, st>>>(d, 1));
  return cudaGetLastError();
}

__global__ void k_mirror_p32(Dev d) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x)
    d.p32[j] = (float)d.p[j];
}

cudaError_t launch_gap_count(const Dev& d, int32_t* slots, cudaStream_t st) {
  const int gb = (int)std::min<int64_t>((d.n + 7) / 8, 8 * (int64_t)(d.sm_count > 0 ? d.sm_count : 148));
  k_gap_count<<<gb, 256, 0, st>>>(d, slots);
  return cudaGetLastError();
}

cudaError_t launch_gap_fill(const Dev& d, cudaStream_t st) {
  const int gb = (int)std::min<int64_t>((d.n + 7) / 8, 8 * (int64_t)(d.sm_count > 0 ? d.sm_count : 148));
  if (d.storage == ST_F32) k_gap_fill<ST_F32><<<gb, 256, 0, st>>>(d);
  else if (d.storage == ST_BF16) k_gap_fill<ST_BF16><<<gb, 256, 0, st>>>(d);
  else k_gap_fill<ST_FP8><<<gb, 256, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_mirror_p32(const Dev& d, const Geo& g, cudaStream_t st) {
  k_mirror_p32<<<g.eN, kBlock, 0, st>>>(d);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- refinement

// Start of a refined Newton step: dx_acc = 0; outer tolerance = the PCG tolerance of the step.
__global__ void k_refine_start(Dev d) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x)
    d.dxr[j] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Scal* sc = d.sc;
    sc->tol2_outer = sc->tol2;
    sc->rr_outer = sc->rhs2;
    sc->refine_it = 0;
    sc->cg_step_total = 0;
    sc->cg_conv_outer = sc->cg_done;   // rhs == 0: nothing to refine
  }
}

// Inner solve setup: dx = 0; PCG tolerance relative to the current FP64 residual in r; the
// inner loop's condition re-armed (a nested loop keeps its last value between outer trips).
__global__ void k_refine_inner(Dev d, cudaGraphConditionalHandle hi, int set_cond) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x)
    d.dx[j] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (set_cond) cudaGraphSetConditional(hi, 1u);
    Scal* sc = d.sc;
    sc->tol2 = sc->refine_eta * sc->refine_eta * sc->rr_outer;
    sc->cg_iter = 0;
    sc->cg_conv = 0;
    sc->cg_done = (sc->rr_outer == 0.0) ? 1 : 0;
  }
}

// dx_acc += dx; p = dx_acc (input of the FP64 operator apply that follows).
__global__ void k_refine_acc(Dev d) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    const double v = d.dxr[j] + d.dx[j];
    d.dxr[j] = v;
    d.p[j] = v;
  }
}

// r = rhs - K dx_acc (q holds K dx_acc from the FP64 operator); ||r||^2; loop condition.
__global__ void k_refine_resid(Dev d, cudaGraphConditionalHandle h, int set_cond) {
  __shared__ double sh[32];
  double rr = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    const double rj = d.rhs[j] - d.q[j];
    d.r[j] = rj;
    rr = fma(rj, rj, rr);
  }
  double v[1] = {rr};
  const int ops[1] = {0};
  double out[1];
  if (grid_reduce<1>(v, ops, d.partials + 27 * kMaxRedBlocks, &d.sc->ticket[T_REF], out, sh)) {
    if (threadIdx.x == 0) {
      Scal* sc = d.sc;
      sc->refine_it += 1;
      sc->cg_step_total += sc->cg_iter;
      sc->rr_outer = out[0];
      sc->rr = out[0];
      const bool ok = isfinite(out[0]);
      if (!ok) sc->status = DS_NUMERICAL;
      sc->cg_conv_outer = ok && out[0] <= sc->tol2_outer;
      const bool cont = ok && !sc->cg_conv_outer && sc->refine_it < sc->refine_max;
      if (set_cond) cudaGraphSetConditional(h, cont ? 1u : 0u);
    }
  }
}

// Fallback when refinement did not reach the tolerance in refine_max passes: plain FP64 PCG
// on the current residual (r = rhs - K dx_acc) to the step's absolute tolerance.  When the
// refinement converged the loop that follows exits at once (cg_done = 1).
__global__ void k_refine_fallback(Dev d) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x)
    d.dx[j] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Scal* sc = d.sc;
    sc->tol2 = sc->tol2_outer;
    sc->cg_iter = 0;
    sc->cg_conv = 0;
    sc->cg_done = (sc->cg_conv_outer || !isfinite(sc->rr_outer) || sc->rr_outer <= sc->tol2_outer) ? 1 : 0;
    sc->fallback = sc->cg_done ? 0 : 1;
  }
}

// End of a refined step: dx = dx_acc (+ the fallback's correction); totals in the PCG fields.
__global__ void k_refine_finish(Dev d) {
  const bool fb = d.sc->fallback;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x)
    d.dx[j] = fb ? d.dxr[j] + d.dx[j] : d.dxr[j];
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Scal* sc = d.sc;
    if (fb) {
      sc->cg_step_total += sc->cg_iter;
      sc->fallback_total += 1;
    } else {
      sc->cg_conv = sc->cg_conv_outer;
      sc->rr = sc->rr_outer;
    }
    sc->cg_iter = sc->cg_step_total;
    sc->tol2 = sc->tol2_outer;
  }
}

// ------------------------------------------------- reduced-precision PCG with replacement
//
// One PCG per Newton step on the reduced-precision operator K~ (FP64 vectors), whose
// recursive residual r is replaced by the true residual rhs - K dx (FP64 operator) whenever it
// has fallen by refine_eta since the last replacement, when it meets the step's tolerance, or
// at the iteration limit; the search direction is kept across replacements (a "reliable
// update" of the residual, Sleijpen and van der Vorst 1996), so the Krylov space built on K~
// is not thrown away as the restarted refinement does.  The step is done when a replaced
// (true) residual meets the tolerance; otherwise the FP64 fallback PCG finishes it.

// Start: tolerance of the step, reference norm = ||rhs||^2 (r = rhs, dx = 0 from the rhs pass).
__global__ void k_ru_start(Dev d) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Scal* sc = d.sc;
    sc->tol2_outer = sc->tol2;
    sc->rr_outer = sc->rhs2;
    sc->rr_ref = sc->rhs2;
    sc->refine_it = 0;
    sc->cg_step_total = 0;
    sc->cg_conv_outer = sc->cg_done;   // rhs == 0: nothing to solve
    sc->ru_do = 0;
    sc->ru_restart = 0;
  }
}

// dx += alpha p; r -= alpha q; ||r||^2; a replacement is asked for when ||r|| fell by
// refine_eta since the last one, met the tolerance, or the iteration limit is reached.
__global__ void k_ru_update(Dev d) {
  __shared__ double sh[32];
  if (d.sc->cg_done) return;
  const double alpha = d.sc->alpha;
  double rr = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    d.dx[j] = fma(alpha, d.p[j], d.dx[j]);
    const double rj = fma(-alpha, d.q[j], d.r[j]);
    d.r[j] = rj;
    rr = fma(rj, rj, rr);
  }
  double v[1] = {rr};
  const int ops[1] = {0};
  double out[1];
  if (grid_reduce<1>(v, ops, d.partials + 17 * kMaxRedBlocks, &d.sc->ticket[T_UPD], out, sh)) {
    if (threadIdx.x == 0) {
      Scal* sc = d.sc;
      sc->cg_iter += 1;
      sc->rr = out[0];
      if (!isfinite(out[0])) {
        sc->cg_done = 1;
        sc->status = DS_NUMERICAL;
        sc->ru_do = 0;
      } else {
        sc->ru_do = (out[0] <= sc->tol2_outer || out[0] <= sc->refine_eta * sc->refine_eta * sc->rr_ref ||
                     sc->cg_iter >= sc->cg_max) ? 1 : 0;
      }
    }
  }
}

// On a replacement (q = K dx from the FP64 operator): r = rhs - q, the new reference norm; the
// step ends when it meets the tolerance (converged) or at the iteration limit.
__global__ void k_ru_resid(Dev d) {
  __shared__ double sh[32];
  if (!d.sc->ru_do) return;
  double rr = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    const double rj = d.rhs[j] - d.q[j];
    d.r[j] = rj;
    rr = fma(rj, rj, rr);
  }
  double v[1] = {rr};
  const int ops[1] = {0};
  double out[1];
  if (grid_reduce<1>(v, ops, d.partials + 27 * kMaxRedBlocks, &d.sc->ticket[T_REF], out, sh)) {
    if (threadIdx.x == 0) {
      Scal* sc = d.sc;
      sc->refine_it += 1;
      sc->rr = out[0];
      // no progress since the last replacement (the true residual fell by less than a tenth:
      // the kept direction has lost conjugacy to the coarse operator's drift): restart the
      // Krylov process from this residual
      sc->ru_restart = out[0] > 0.81 * sc->rr_outer ? 1 : 0;
      sc->rr_ref = out[0];
      sc->rr_outer = out[0];
      if (!isfinite(out[0])) {
        sc->status = DS_NUMERICAL;
        sc->cg_done = 1;
      } else if (out[0] <= sc->tol2_outer) {
        sc->cg_done = 1;
        sc->cg_conv = 1;
        sc->cg_conv_outer = 1;
      } else if (sc->cg_iter >= sc->cg_max) {
        sc->cg_done = 1;
      }
    }
  }
}

// Preconditioned residual after the (possibly replaced) r.  ZM 0 (Jacobi): z = r / M, r^T z,
// beta.  ZM 1 (Jacobi + low rank): z0 = r / M, the low-rank correction follows.
template <int ZM>
__global__ void k_ru_z(Dev d) {
  __shared__ double sh[32];
  if (d.sc->cg_done) return;
  double rz = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    const double zj = d.r[j] * d.Minv[j];
    d.z[j] = zj;
    rz = fma(d.r[j], zj, rz);
  }
  if (ZM == 1) return;
  double v[1] = {rz};
  const int ops[1] = {0};
  double out[1];
  if (grid_reduce<1>(v, ops, d.partials + 29 * kMaxRedBlocks, &d.sc->ticket[T_CORR], out, sh)) {
    if (threadIdx.x == 0) {
      Scal* sc = d.sc;
      sc->beta = out[0] / sc->rz;
      sc->rz = out[0];
    }
  }
}

// After a replacement that made no progress: p = z (beta = 0), a fresh Krylov start.
__global__ void k_ru_restart(Dev d) {
  Scal* sc = d.sc;
  if (sc->ru_restart) {
    sc->beta = 0.0;
    sc->ru_restart = 0;
  }
}

// End: the step so far in dxr (the FP64 fallback adds its correction to it), PCG totals.
__global__ void k_ru_end(Dev d) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x)
    d.dxr[j] = d.dx[j];
  if (blockIdx.x == 0 && threadIdx.x == 0) d.sc->cg_step_total = d.sc->cg_iter;
}

cudaError_t launch_ru_start(const Dev& d, cudaStream_t st) {
  k_ru_start<<<1, 32, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_apply_ru(const Dev& d, const Geo& g, cudaStream_t st);   // kernels.cu

// One trip of the replacement PCG: q = K~ p, the update, the FP64 replacement when asked for,
// the preconditioner, the next direction (k_cg_p sets the loop condition).
cudaError_t launch_ru_body(const Dev& d, const Geo& g, int precond, cudaGraphConditionalHandle h, cudaStream_t st,
                           bool in_graph) {
  cudaError_t e = launch_op_lp(d, g, st);
  if (e != cudaSuccess) return e;
  k_ru_update<<<g.eN, kBlock, 0, st>>>(d);
  e = launch_apply_ru(d, g, st);
  if (e != cudaSuccess) return e;
  k_ru_resid<<<g.eN, kBlock, 0, st>>>(d);
  if (precond == PC_JACOBI_LR) {
    k_ru_z<1><<<g.eN, kBlock, 0, st>>>(d);
    e = launch_stiff_apply(d, g, st);
    if (e != cudaSuccess) return e;
  } else {
    k_ru_z<0><<<g.eN, kBlock, 0, st>>>(d);
  }
  k_ru_restart<<<1, 1, 0, st>>>(d);
  return launch_cg_p(d, g, h, in_graph, st);
}

cudaError_t launch_ru_end(const Dev& d, const Geo& g, cudaStream_t st) {
  k_ru_end<<<g.eN, kBlock, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_refine_start(const Dev& d, const Geo& g, cudaStream_t st) {
  k_refine_start<<<g.eN, kBlock, 0, st>>>(d);
  return cudaGetLastError();
}
cudaError_t launch_refine_inner(const Dev& d, const Geo& g, cudaGraphConditionalHandle hi, cudaStream_t st) {
  k_refine_inner<<<g.eN, kBlock, 0, st>>>(d, hi, hi != 0 ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t launch_refine_tail(const Dev& d, const Geo& g, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_refine_acc<<<g.eN, kBlock, 0, st>>>(d);
  cudaError_t e = launch_apply(d, g, st);        // FP64 operator: q = K dx_acc
  if (e != cudaSuccess) return e;
  k_refine_resid<<<g.eN, kBlock, 0, st>>>(d, h, h != 0 ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t launch_refine_fallback(const Dev& d, const Geo& g, cudaStream_t st) {
  k_refine_fallback<<<g.eN, kBlock, 0, st>>>(d);
  return cudaGetLastError();
}
cudaError_t launch_refine_finish(const Dev& d, const Geo& g, cudaStream_t st) {
  k_refine_finish<<<g.eN, kBlock, 0, st>>>(d);
  return cudaGetLastError();
}

}  // namespace ipmk
