// Double-float PCG operator and the runs of R's rows.
//
// GB300 issues two float64 fused multiply-adds per SM per clock: at the RT size the FP64
// operator passes (one multiply-add per stored entry) are bound by that pipe before HBM.  The
// double-float passes carry every value of R, R^T, p and v as a (hi, lo) pair of float32 (the
// same 8 bytes as the double) and form each product and the row sums with error-free
// transformations on the float32 pipe (common.cuh), which is 64 times wider, leaving HBM as
// the bound.  The row sums are exact to about 2^-44 relative to sum |a x| (48-bit operands,
// compensated sums), far below the smallest PCG tolerance; the operator stays exactly
// symmetric (the column pass forms R^T diag(omega) R with the same stored values as the rows
// pass, and every sum has a fixed order), so conjugate gradients remain valid.  Residuals,
// the start point, the right-hand side and the preconditioner keep the FP64 copies.
//
// Runs: the columns of a dose row come in a few contiguous spot bands.  A run is a maximal
// stretch of consecutive stored entries of a row whose columns increase by one; runs are cut
// into pieces of at most 32 entries, and the rows pass over pieces reads one 8-byte
// descriptor per piece instead of one int32 index per entry, with the values and the gathers
// of p at consecutive addresses and no load waiting for an index.
#include "state.h"

namespace ipmk {

static __device__ __forceinline__ int gwarp_d() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
static __device__ __forceinline__ int nwarps_d() { return (gridDim.x * blockDim.x) >> 5; }

#define FOR_GROUP_ROWS_D(G, r, ok, nrows)                                                                    \
  for (int64_t r##_0 = (int64_t)gwarp_d() * (32 / G); r##_0 < (nrows); r##_0 += (int64_t)nwarps_d() * (32 / G)) \
    for (int64_t r = r##_0 + (threadIdx.x & 31) / G, r##_once = 0; r##_once == 0; r##_once = 1)               \
      for (bool ok = r < (nrows), ok##_once = true; ok##_once; ok##_once = false)

#define DISPATCH_GD(g, ...)                                  \
  switch (g) {                                               \
    case 4: { constexpr int G = 4; __VA_ARGS__; } break;     \
    case 8: { constexpr int G = 8; __VA_ARGS__; } break;     \
    case 16: { constexpr int G = 16; __VA_ARGS__; } break;   \
    default: { constexpr int G = 32; __VA_ARGS__; } break;   \
  }

// ---------------------------------------------------------------- set-up

// out = (hi, lo) pairs of a; *flag |= 1 if a non-zero value lies outside [2^-90, 2^90], where
// the pair would lose bits to the float32 exponent range (the caller then keeps FP64).
__global__ void k_df_split(const double* __restrict__ a, float2* __restrict__ out, int64_t n, int* flag) {
  bool bad = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = a[e];
    const double av = fabs(v);
    if (v != 0.0 && !(av >= 0x1p-90 && av <= 0x1p90)) bad = true;
    out[e] = df_split(v);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

cudaError_t launch_df_split(const Dev& d, int* out_of_range, cudaStream_t st) {
  if (!d.R_df || d.nnzR == 0) return cudaSuccess;
  const int gb = (int)std::min<int64_t>((d.nnzR + 255) / 256, 8 * (int64_t)(d.sm_count > 0 ? d.sm_count : 148));
  k_df_split<<<gb, 256, 0, st>>>(d.R_val, const_cast<float2*>(d.R_df), d.nnzR, out_of_range);
  k_df_split<<<gb, 256, 0, st>>>(d.RT_val, const_cast<float2*>(d.RT_df), d.nnzR, out_of_range);
  return cudaGetLastError();
}

__global__ void k_mirror_df(Dev d) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x)
    d.p_df[j] = df_split(d.p[j]);
}

cudaError_t launch_mirror_df(const Dev& d, const Geo& g, cudaStream_t st) {
  k_mirror_df<<<g.eN, kBlock, 0, st>>>(d);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- row sums

// Double-float dot of one CSR row with a double-float vector by a group of G lanes (lane gl
// takes entries gl, gl + G, ...; two in flight), summed over the group.
template <int G>
__device__ __forceinline__ void group_row_mac_df(const int64_t beg, const int64_t end, const int gl,
                                                 const int32_t* __restrict__ idx, const float2* __restrict__ val,
                                                 const float2* __restrict__ x, float& h, float& l) {
  int64_t e = beg + gl;
  for (; e + 3 * G < end; e += 4 * G) {
    const float2 a0 = __ldg(val + e), a1 = __ldg(val + e + G), a2 = __ldg(val + e + 2 * G), a3 = __ldg(val + e + 3 * G);
    const int i0 = __ldg(idx + e), i1 = __ldg(idx + e + G), i2 = __ldg(idx + e + 2 * G), i3 = __ldg(idx + e + 3 * G);
    const float2 x0 = __ldg(x + i0), x1 = __ldg(x + i1), x2 = __ldg(x + i2), x3 = __ldg(x + i3);
    df_mac(a0, x0, h, l);
    df_mac(a1, x1, h, l);
    df_mac(a2, x2, h, l);
    df_mac(a3, x3, h, l);
  }
  for (; e < end; e += G) df_mac(__ldg(val + e), __ldg(x + __ldg(idx + e)), h, l);
}

// ---------------------------------------------------------------- operator passes

// v = omega o (R p), double-float products, v stored as pairs.  MODE 0: inside PCG (skips once
// converged; the doubly augmented system's bottom block as in the FP64 pass); MODE 1: one apply.
template <int MODE, int G, bool RUNS>
__global__ void __launch_bounds__(256, 6) k_op_rows_df(Dev d) {
  if (MODE == 0 && d.sc->cg_done) return;
  const int gl = threadIdx.x & (G - 1);
  FOR_GROUP_ROWS_D(G, ri, ok, d.nR) {
    const int64_t r = (ok && d.rperm) ? (int64_t)d.rperm[ri] : ri;
    float th = 0.f, tl = 0.f;
    if (RUNS) {
      for_row_pieces<G>(d, r, ok, gl, [&](int64_t e, int c) { df_mac(__ldg(d.R_df + e), __ldg(d.p_df + c), th, tl); });
    } else {
      const int64_t beg = ok ? d.R_ptr[r] : 0, end = ok ? d.R_ptr[r + 1] : 0;
      group_row_mac_df<G>(beg, end, gl, d.R_idx, d.R_df, d.p_df, th, tl);
    }
    df_group_pair<G>(th, tl);
    if (ok && gl == 0) {
      if (MODE == 0 && d.aug) {
        const double t = df_value(th, tl);
        double v = d.omega[r] * t;
        const int32_t k = d.rowk[r];
        if (k >= 0) {
          const double pb = d.p[d.n + k];
          v -= pb;
          d.q[d.n + k] = -t + pb * (d.s[k] / d.y[k]);
        }
        d.v_df[r] = df_split(v);
      } else {
        // v = omega t as a double-float product (no float64 arithmetic per row)
        const float2 w = df_split(d.omega[r]);
        float vh = 0.f, vl = 0.f;
        df_mac(w, make_float2(th, tl), vh, vl);
        float s, e;
        two_sum(vh, vl, s, e);
        d.v_df[r] = make_float2(s, e);
      }
    }
  }
}

// q = R^T v + Hs p + U (W t) + (h0 + sigma) o p with the R^T v sums in double-float; p^T q ->
// alpha = rz / p^T q (last block), exactly as the FP64 column pass.
template <int MODE, int G>
__global__ void __launch_bounds__(256, 6) k_op_cols_df(Dev d) {
  __shared__ double sh[32];
  if (MODE == 0 && d.sc->cg_done) return;
  const int gl = threadIdx.x & (G - 1);
  double pq = 0.0;
  FOR_GROUP_ROWS_D(G, j, ok, d.n) {
    const int64_t beg = ok ? d.RT_ptr[j] : 0, end = ok ? d.RT_ptr[j + 1] : 0;
    float ah = 0.f, al = 0.f;
    group_row_mac_df<G>(beg, end, gl, d.RT_idx, d.RT_df, d.v_df, ah, al);
    df_group_pair<G>(ah, al);
    double acc = gl == 0 ? df_value(ah, al) : 0.0;   // float64 once per row (lane 0 keeps it)
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

cudaError_t launch_op_rows_df(const Dev& d, const Geo& g, int mode, cudaStream_t st) {
  if (!d.nR) return cudaSuccess;
  if (d.ntiles) return launch_op_rows_staged(d, mode, st);
  if (d.runs) {
    if (mode == 0) { DISPATCH_GD(d.g_rows, k_op_rows_df<0, G, true><<<g.gRc, kBlock, 0, st>>>(d)); }
    else { DISPATCH_GD(d.g_rows, k_op_rows_df<1, G, true><<<g.gRc, kBlock, 0, st>>>(d)); }
  } else {
    if (mode == 0) { DISPATCH_GD(d.g_rows, k_op_rows_df<0, G, false><<<g.gRc, kBlock, 0, st>>>(d)); }
    else { DISPATCH_GD(d.g_rows, k_op_rows_df<1, G, false><<<g.gRc, kBlock, 0, st>>>(d)); }
  }
  return cudaGetLastError();
}

cudaError_t launch_op_cols_df(const Dev& d, const Geo& g, int mode, cudaStream_t st) {
  if (mode == 0) { DISPATCH_GD(d.g_cols, k_op_cols_df<0, G><<<g.gNc, kBlock, 0, st>>>(d)); }
  else { DISPATCH_GD(d.g_cols, k_op_cols_df<1, G><<<g.gNc, kBlock, 0, st>>>(d)); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- runs of R's rows

// An entry starts a run if it is the first of its row or its column is not one more than the
// previous entry's; a run of L entries is cut into ceil(L / kPiece) pieces.  One warp per row
// walks the run starts found by a ballot over each 32-entry stretch (the same walk in every
// lane).  EMIT 0: count runs and pieces per row; EMIT 1: write the piece descriptors.
template <int EMIT>
__global__ void k_runs_walk(Dev d, int32_t* __restrict__ nruns, int32_t* __restrict__ npieces) {
  const int lane = threadIdx.x & 31;
  int32_t* pcol = const_cast<int32_t*>(d.pc_col);
  uint32_t* pol = const_cast<uint32_t*>(d.pc_ol);
  for (int64_t r = gwarp_d(); r < d.nR; r += nwarps_d()) {
    const int64_t beg = d.R_ptr[r], end = d.R_ptr[r + 1];
    int64_t cur = beg;                           // first entry of the open run
    int64_t k = EMIT ? d.pc_ptr[r] : 0;          // next piece slot
    int nr = 0, np = 0;
    auto close = [&](int64_t stop) {             // the run [cur, stop) -> its pieces
      const int32_t c0 = d.R_idx[cur];
      for (int64_t s = cur; s < stop; s += kPiece) {
        const int64_t len = stop - s < kPiece ? stop - s : kPiece;
        if (EMIT && lane == 0) {
          pcol[k] = c0 + (int32_t)(s - cur);
          pol[k] = ((uint32_t)(s - beg) << 6) | (uint32_t)len;
        }
        ++k;
        ++np;
      }
    };
    for (int64_t e0 = beg; e0 < end; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool start = e < end && (e == beg || d.R_idx[e] != d.R_idx[e - 1] + 1);
      unsigned m = __ballot_sync(0xffffffffu, start);
      while (m) {
        const int64_t pos = e0 + (__ffs(m) - 1);
        m &= m - 1;
        if (pos > beg) close(pos);
        cur = pos;
        ++nr;
      }
    }
    if (end > beg) close(end);
    if (!EMIT && lane == 0) {
      nruns[r] = nr;
      npieces[r] = np;
    }
  }
}

cudaError_t launch_runs_count(const Dev& d, int32_t* runs, int32_t* pieces, cudaStream_t st) {
  if (!d.nR) return cudaSuccess;
  const int gb = (int)std::min<int64_t>((d.nR + 7) / 8, 8 * (int64_t)(d.sm_count > 0 ? d.sm_count : 148));
  k_runs_walk<0><<<gb, 256, 0, st>>>(d, runs, pieces);
  return cudaGetLastError();
}

cudaError_t launch_runs_fill(const Dev& d, cudaStream_t st) {
  if (!d.nR) return cudaSuccess;
  const int gb = (int)std::min<int64_t>((d.nR + 7) / 8, 8 * (int64_t)(d.sm_count > 0 ? d.sm_count : 148));
  k_runs_walk<1><<<gb, 256, 0, st>>>(d, nullptr, nullptr);
  return cudaGetLastError();
}

}  // namespace ipmk
