// Rows pass of the PCG operator with the matrix values streamed into shared memory by the
// bulk-copy (TMA) engine.
//
// R's rows are grouped into tiles: consecutive rows whose values take at most kStageBytes
// (a row longer than that is a tile of its own and is read from global memory).  One block of
// kStagedThreads threads per SM runs a three-stage pipeline over its tiles (tile t goes to
// block t mod gridDim): thread 0 arms the stage's mbarrier with the tile's byte count and
// issues cp.async.bulk copies of the tile's values (16-byte aligned, whole 16-byte units)
// into the stage; the threads wait on the barrier's phase, compute the tile's rows from
// shared memory (pieces of runs: one descriptor per piece from global memory, the gathered
// vector from L1/L2), meet at a block barrier, and thread 0 refills the stage with the tile
// three ahead.  The copy engine keeps two tiles in flight per SM while one is computed, so
// the value stream no longer waits on load latency.
//
// Every wait is bounded (options.wait_limit_ms, measured on the global timer): when it runs
// out, the block records DS_TIMEOUT, stops the PCG loop, waits (bounded again) for the
// copies it has issued, and returns; the host reports IPM_ERR_TIMEOUT.  options.wait_test
// arms the first tile's barrier for 16 bytes more than is copied, so that wait runs out with
// every copy landed (the test of this path).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "state.h"

namespace ipmk {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

// One arrival plus the byte count the phase waits for.
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity to complete, at most limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

// nbytes (a multiple of 16) from global src (16-byte aligned) to shared dst (16-byte aligned),
// completing on the barrier; called by one thread.
__device__ __forceinline__ void bulk_copy(uint32_t dst, const char* src, uint32_t nbytes, uint32_t bar) {
  constexpr uint32_t kChunk = 32768;
  for (uint32_t off = 0; off < nbytes; off += kChunk) {
    const uint32_t sz = nbytes - off < kChunk ? nbytes - off : kChunk;
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst + off),
                 "l"(src + off), "r"(sz), "r"(bar)
                 : "memory");
  }
}

// Value types of the staged passes: double-float pairs (the FP64-storage operator) or the
// reduced-precision copies.
template <int K> struct Val;
template <> struct Val<ST_F64> {   // double-float pairs
  static constexpr int B = 8;
};
template <> struct Val<ST_F32> {
  static constexpr int B = 4;
  static __device__ __forceinline__ float dec(const char* p) { return *reinterpret_cast<const float*>(p); }
};
template <> struct Val<ST_BF16> {
  static constexpr int B = 2;
  static __device__ __forceinline__ float dec(const char* p) {
    return __uint_as_float((uint32_t)(*reinterpret_cast<const unsigned short*>(p)) << 16);
  }
};
template <> struct Val<ST_FP8> {
  static constexpr int B = 1;
  static __device__ __forceinline__ float dec(const char* p) {
    return static_cast<float>(*reinterpret_cast<const __nv_fp8_e4m3*>(p));
  }
};

// Bytes [lo, hi) of the tile's values: whole 16-byte units around its entries.
template <int K>
__device__ __forceinline__ void tile_span(const Dev& d, int64_t t, int64_t& r0, int64_t& r1, uint64_t& lo,
                                          uint64_t& hi) {
  r0 = d.tile_row[t];
  r1 = d.tile_row[t + 1];
  const uint64_t e0 = (uint64_t)d.R_ptr[r0], e1 = (uint64_t)d.R_ptr[r1];
  lo = (e0 * Val<K>::B) & ~(uint64_t)15;
  hi = (e1 * Val<K>::B + 15) & ~(uint64_t)15;
}

template <int K>
__device__ __forceinline__ const char* values_of(const Dev& d) {
  return K == ST_F64 ? reinterpret_cast<const char*>(d.R_df) : static_cast<const char*>(d.Rq);
}

// Thread 0: arms stage s for tile t and issues its copies (none for a tile read from global
// memory, whose phase completes at the arrival).  Returns the bytes it asked for.
template <int K>
__device__ __forceinline__ void issue_tile(const Dev& d, int64_t t, char* stage, uint32_t bar, bool plant) {
  int64_t r0, r1;
  uint64_t lo, hi;
  tile_span<K>(d, t, r0, r1, lo, hi);
  const uint64_t nb = hi - lo;
  if (nb > (uint64_t)kStageBytes + 16) {
    mbar_expect(bar, 0);
    return;
  }
  mbar_expect(bar, (uint32_t)nb + (plant ? 16u : 0u));
  bulk_copy(smem_u32(stage), values_of<K>(d) + lo, (uint32_t)nb, bar);
}

}  // namespace

// Staged rows pass.  K = ST_F64: v = omega o (R p) in double-float (MODE 0 inside PCG, with
// the doubly augmented bottom block; MODE 1 one apply).  K = reduced storage: w32 = s^2
// (w_R + thR) o (R~ p32) (MODE 0 inside PCG, MODE 1 standalone).
template <int K, int MODE, int G>
__global__ void __launch_bounds__(kStagedThreads, 1) k_op_rows_staged(Dev d) {
  extern __shared__ __align__(128) char smem[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ int s_skip;
  const int tid = threadIdx.x;
  // one read of the PCG flag for the whole block (another block may set it while this one
  // starts, and every thread must take the same path through the block barriers)
  if (tid == 0) s_skip = (MODE == 0) ? d.sc->cg_done : 0;
  __syncthreads();
  if (s_skip) return;
  const int gl = tid & (G - 1), grp = tid / G, ngroups = kStagedThreads / G;
  const int64_t nt = d.ntiles;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&bars[s]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto stage_of = [&](int s) { return smem + (size_t)s * kStageAlloc; };
  if (tid == 0)
    for (int s = 0; s < kStages; ++s) {
      const int64_t t = blockIdx.x + (int64_t)s * gridDim.x;
      if (t < nt) issue_tile<K>(d, t, stage_of(s), smem_u32(&bars[s]), d.wait_test && t == 0);
    }
  int64_t i = 0;
  bool bad = false;   // the same in every thread: decided by a block-wide vote
  for (;; ++i) {
    const int64_t t = blockIdx.x + i * gridDim.x;
    if (t >= nt) break;
    const int s = (int)(i % kStages);
    const uint32_t parity = (uint32_t)((i / kStages) & 1);
    const bool ok_wait = mbar_wait(smem_u32(&bars[s]), parity, d.wait_ns);
    if (!__syncthreads_and(ok_wait)) {
      bad = true;
      break;
    }
    int64_t r0, r1;
    uint64_t lo, hi;
    tile_span<K>(d, t, r0, r1, lo, hi);
    const bool direct = hi - lo > (uint64_t)kStageBytes + 16;
    const char* sv = stage_of(s);
    const char* gv = values_of<K>(d);
    for (int64_t k0 = 0; k0 < r1 - r0; k0 += ngroups) {
      const int64_t r = r0 + k0 + grp;
      const bool ok = r < r1;
      if constexpr (K == ST_F64) {
        float th = 0.f, tl = 0.f;
        for_row_pieces<G>(d, r, ok, gl, [&](int64_t e, int c) {
          const uint64_t b = (uint64_t)e * 8;
          const float2 a = direct ? __ldg(reinterpret_cast<const float2*>(gv + b))
                                  : *reinterpret_cast<const float2*>(sv + (b - lo));
          df_mac(a, __ldg(d.p_df + c), th, tl);
        });
        df_group_pair<G>(th, tl);
        if (ok && gl == 0) {
          if (MODE == 0 && d.aug) {
            const double tv = df_value(th, tl);
            double v = d.omega[r] * tv;
            const int32_t k = d.rowk[r];
            if (k >= 0) {
              const double pb = d.p[d.n + k];
              v -= pb;
              d.q[d.n + k] = -tv + pb * (d.s[k] / d.y[k]);
            }
            d.v_df[r] = df_split(v);
          } else {
            const float2 w = df_split(d.omega[r]);
            float vh = 0.f, vl = 0.f;
            df_mac(w, make_float2(th, tl), vh, vl);
            float hs, ls;
            two_sum(vh, vl, hs, ls);
            d.v_df[r] = make_float2(hs, ls);
          }
        }
      } else {
        float a = 0.f;
        for_row_pieces<G>(d, r, ok, gl, [&](int64_t e, int c) {
          const uint64_t b = (uint64_t)e * Val<K>::B;
          const float v = Val<K>::dec(direct ? gv + b : sv + (b - lo));
          a = fmaf(v, __ldg(d.p32 + c), a);
        });
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (ok && gl == 0) {
          const double sc = (double)d.scaleR[r];
          d.w32[r] = (float)((d.wR[r] + d.thR[r]) * sc * sc * (double)a);
        }
      }
    }
    __syncthreads();   // every thread is done with stage s
    if (tid == 0) {
      const int64_t tn = t + (int64_t)kStages * gridDim.x;
      if (tn < nt) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_tile<K>(d, tn, stage_of(s), smem_u32(&bars[s]), false);
      }
    }
  }
  if (bad) {
    // a wait ran out: stop the PCG loop, then wait (bounded) for the copies still issued
    if (tid == 0) {
      d.sc->status = DS_TIMEOUT;
      d.sc->cg_done = 1;
      for (int64_t j = i; j < i + kStages; ++j) {
        const int64_t t = blockIdx.x + j * gridDim.x;
        if (t >= nt) break;
        mbar_wait(smem_u32(&bars[j % kStages]), (uint32_t)((j / kStages) & 1), d.wait_ns);
      }
    }
    __syncthreads();
  }
}

#define DISPATCH_GS(g, ...)                                  \
  switch (g) {                                               \
    case 8: { constexpr int G = 8; __VA_ARGS__; } break;     \
    case 16: { constexpr int G = 16; __VA_ARGS__; } break;   \
    default: { constexpr int G = 32; __VA_ARGS__; } break;   \
  }

static int staged_grid(const Dev& d) {
  const int64_t sm = d.sm_count > 0 ? d.sm_count : 148;
  return (int)std::max<int64_t>(1, std::min<int64_t>(d.ntiles, sm));
}

template <int K>
static void launch_staged_k(const Dev& d, int mode, cudaStream_t st) {
  const int grid = staged_grid(d);
  const size_t smem = (size_t)kStages * kStageAlloc;
  // lanes per row: 8, 16 or 32 (the staged tiles hold 1-4 rows per group; 4 lanes are not offered)
  const int g = d.g_rows < 8 ? 8 : d.g_rows;
  if (mode == 0) { DISPATCH_GS(g, k_op_rows_staged<K, 0, G><<<grid, kStagedThreads, smem, st>>>(d)); }
  else { DISPATCH_GS(g, k_op_rows_staged<K, 1, G><<<grid, kStagedThreads, smem, st>>>(d)); }
}

cudaError_t launch_op_rows_staged(const Dev& d, int mode, cudaStream_t st) {
  if (!d.nR || !d.ntiles) return cudaSuccess;
  if (d.df) launch_staged_k<ST_F64>(d, mode, st);
  else if (d.storage == ST_F32) launch_staged_k<ST_F32>(d, mode, st);
  else if (d.storage == ST_BF16) launch_staged_k<ST_BF16>(d, mode, st);
  else launch_staged_k<ST_FP8>(d, mode, st);
  return cudaGetLastError();
}

cudaError_t prepare_staged() {
  cudaError_t e = cudaSuccess;
  const int smem = kStages * kStageAlloc;
  auto set = [&](const void* f) {
    const cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (r != cudaSuccess && e == cudaSuccess) e = r;
  };
#define IPMK_SET_STAGED(K)                                                                              \
  set((const void*)k_op_rows_staged<K, 0, 8>); set((const void*)k_op_rows_staged<K, 0, 16>);            \
  set((const void*)k_op_rows_staged<K, 0, 32>); set((const void*)k_op_rows_staged<K, 1, 8>);            \
  set((const void*)k_op_rows_staged<K, 1, 16>); set((const void*)k_op_rows_staged<K, 1, 32>);
  IPMK_SET_STAGED(ST_F64)
  IPMK_SET_STAGED(ST_F32)
  IPMK_SET_STAGED(ST_BF16)
  IPMK_SET_STAGED(ST_FP8)
#undef IPMK_SET_STAGED
  return e;
}

}  // namespace ipmk
