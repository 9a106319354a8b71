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

// Layout of one stage: the tile's values, its pieces' descriptors (columns, offset/length
// words) and the row and piece pointers of its rows, each copied as whole 16-byte units.
constexpr int al16(int x) { return (x + 15) & ~15; }
struct StageLayout {
  static constexpr int kVal = 0;
  static constexpr int kCol = kVal + al16(kStageValBytes + 16);
  static constexpr int kOl = kCol + al16(4 * kStagePieces + 16);
  static constexpr int kRp = kOl + al16(4 * kStagePieces + 16);
  static constexpr int kPp = kRp + al16(8 * (kStageRows + 1) + 16);
  static constexpr int kEnd = kPp + al16(8 * (kStageRows + 1) + 16);
};
static_assert(StageLayout::kEnd <= kStageAlloc, "stage layout exceeds the stage");
static_assert(StageLayout::kCol % 16 == 0 && StageLayout::kOl % 16 == 0 && StageLayout::kRp % 16 == 0 &&
              StageLayout::kPp % 16 == 0, "stage sections must start on 16-byte boundaries");

// One staged array section: bytes [lo, hi) of the global array, rounded out to 16 bytes.
struct Span {
  uint64_t lo, hi;
};
__device__ __forceinline__ Span span_of(uint64_t first, uint64_t end, uint64_t elem) {
  return Span{(first * elem) & ~(uint64_t)15, (end * elem + 15) & ~(uint64_t)15};
}

// The spans of tile t: values of its entries, descriptors of its pieces, pointers of its rows.
template <int K>
struct TileSpans {
  int64_t r0, r1, k0, k1, e0, e1;
  Span v, c, o, rp, pp;
  bool direct;   // too large for a stage: read from global memory
  __device__ __forceinline__ TileSpans(const Dev& d, int64_t t) {
    r0 = d.tile_row[t];
    r1 = d.tile_row[t + 1];
    e0 = d.R_ptr[r0];
    e1 = d.R_ptr[r1];
    k0 = d.pc_ptr[r0];
    k1 = d.pc_ptr[r1];
    v = span_of(e0, e1, Val<K>::B);
    c = span_of(k0, k1, 4);
    o = span_of(k0, k1, 4);
    rp = span_of(r0, r1 + 1, 8);
    pp = span_of(r0, r1 + 1, 8);
    direct = v.hi - v.lo > (uint64_t)kStageValBytes + 16 || (k1 - k0) > kStagePieces || (r1 - r0) > kStageRows;
  }
  __device__ __forceinline__ uint32_t bytes() const {
    return (uint32_t)((v.hi - v.lo) + (c.hi - c.lo) + (o.hi - o.lo) + (rp.hi - rp.lo) + (pp.hi - pp.lo));
  }
};

template <int K>
__device__ __forceinline__ const char* values_of(const Dev& d) {
  return K == ST_F64 ? reinterpret_cast<const char*>(d.R_df) : static_cast<const char*>(d.Rq);
}

// Thread 0: arms stage s for tile t and issues its copies (none for a tile read from global
// memory, whose phase completes at the arrival).  plant: 16 bytes more are expected than copied.
template <int K>
__device__ __forceinline__ void issue_tile(const Dev& d, int64_t t, char* stage, uint32_t bar, bool plant) {
  const TileSpans<K> ts(d, t);
  if (ts.direct) {
    mbar_expect(bar, 0);
    return;
  }
  mbar_expect(bar, ts.bytes() + (plant ? 16u : 0u));
  const uint32_t st = smem_u32(stage);
  bulk_copy(st + StageLayout::kVal, values_of<K>(d) + ts.v.lo, (uint32_t)(ts.v.hi - ts.v.lo), bar);
  bulk_copy(st + StageLayout::kCol, reinterpret_cast<const char*>(d.pc_col) + ts.c.lo, (uint32_t)(ts.c.hi - ts.c.lo), bar);
  bulk_copy(st + StageLayout::kOl, reinterpret_cast<const char*>(d.pc_ol) + ts.o.lo, (uint32_t)(ts.o.hi - ts.o.lo), bar);
  bulk_copy(st + StageLayout::kRp, reinterpret_cast<const char*>(d.R_ptr) + ts.rp.lo, (uint32_t)(ts.rp.hi - ts.rp.lo), bar);
  bulk_copy(st + StageLayout::kPp, reinterpret_cast<const char*>(d.pc_ptr) + ts.pp.lo, (uint32_t)(ts.pp.hi - ts.pp.lo), bar);
}

// Lanes per row of the staged passes: 16 for double-float (a tile holds up to 32 rows, one per
// group of the 512 threads), 8 for the narrow storages (up to 64 rows).
template <int K> struct StagedLanes { static constexpr int G = K == ST_F64 ? 16 : 8; };

}  // namespace

// Staged rows pass.  K = ST_F64: v = omega o (R p) in double-float (MODE 0 inside PCG, with
// the doubly augmented bottom block; MODE 1 one apply).  K = reduced storage: w32 = s^2
// (w_R + thR) o (R~ p32) (MODE 0 inside PCG, MODE 1 standalone).
//
// Each group of G lanes takes one row of the tile; per chunk of NP pieces every lane first
// issues its 16 gathers of the vector (and reads the 16 values from the stage), then does the
// 16 multiply-adds in four independent chains, so the gathers of a lane are in flight together.
template <int K, int MODE>
__global__ void __launch_bounds__(kStagedThreads, 1) k_op_rows_staged(Dev d) {
  constexpr int G = StagedLanes<K>::G;
  constexpr int PP = kPiece / G;    // positions of a piece per lane
  constexpr int NP = 16 / PP;       // pieces per chunk: 16 entries per lane
  extern __shared__ __align__(128) char smem[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ int s_skip;
  const int tid = threadIdx.x;
  // one read of the PCG flag for the whole block (another block may set it while this one
  // starts, and every thread must take the same path through the block barriers)
  if (tid == 0) s_skip = (MODE == 0) ? d.sc->cg_done : 0;
  __syncthreads();
  if (s_skip) return;
  const int gl = tid & (G - 1), grp = tid / G;
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
  const char* gv = values_of<K>(d);
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
    const TileSpans<K> ts(d, t);
    const char* st = stage_of(s);
    const int32_t* scol = reinterpret_cast<const int32_t*>(st + StageLayout::kCol);
    const uint32_t* sol = reinterpret_cast<const uint32_t*>(st + StageLayout::kOl);
    const int64_t* srp = reinterpret_cast<const int64_t*>(st + StageLayout::kRp);
    const int64_t* spp = reinterpret_cast<const int64_t*>(st + StageLayout::kPp);
    const int64_t kc = (int64_t)(ts.c.lo / 4), kr = (int64_t)(ts.rp.lo / 8);   // first staged element
    for (int64_t q0 = 0; q0 < ts.r1 - ts.r0; q0 += kStagedThreads / G) {
      const int64_t r = ts.r0 + q0 + grp;
      const bool ok = r < ts.r1;
      int64_t rb = 0, kb = 0, ke = 0;
      if (ok) {
        rb = ts.direct ? d.R_ptr[r] : srp[r - kr];
        kb = ts.direct ? d.pc_ptr[r] : spp[r - kr];
        ke = ts.direct ? d.pc_ptr[r + 1] : spp[r + 1 - kr];
      }
      const unsigned np = (unsigned)(ke - kb);
      const unsigned npmax = __reduce_max_sync(0xffffffffu, np);
      if constexpr (K == ST_F64) {
        float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
        for (unsigned c0 = 0; c0 < npmax; c0 += NP) {
          float2 av[NP * PP], xv[NP * PP];
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            const int64_t k = kb + c0 + q;
            const bool valid = c0 + q < np;
            const int col = valid ? (ts.direct ? d.pc_col[k] : scol[k - kc]) : 0;
            const uint32_t ol = valid ? (ts.direct ? d.pc_ol[k] : sol[k - kc]) : 0u;
            const int len = (int)(ol & 63u);
            const int64_t eb = rb + (int64_t)(ol >> 6);
#pragma unroll
            for (int u = 0; u < PP; ++u) {
              const int j = gl + u * G;
              const bool in = j < len;
              const uint64_t b = (uint64_t)(eb + j) * 8;
              xv[q * PP + u] = in ? __ldg(d.p_df + col + j) : make_float2(0.f, 0.f);
              av[q * PP + u] = !in ? make_float2(0.f, 0.f)
                               : ts.direct ? __ldg(reinterpret_cast<const float2*>(gv + b))
                                           : *reinterpret_cast<const float2*>(st + StageLayout::kVal + (b - ts.v.lo));
            }
          }
#pragma unroll
          for (int u = 0; u < NP * PP; ++u) df_mac(av[u], xv[u], h[u & 3], l[u & 3]);
        }
        // the four chains, then the group, in a fixed order
        float th = h[0], tl = l[0];
#pragma unroll
        for (int c = 1; c < 4; ++c) {
          float s2, e2;
          two_sum(th, h[c], s2, e2);
          th = s2;
          tl = __fadd_rn(__fadd_rn(tl, l[c]), e2);
        }
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
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (unsigned c0 = 0; c0 < npmax; c0 += NP) {
          float av[NP * PP], xv[NP * PP];
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            const int64_t k = kb + c0 + q;
            const bool valid = c0 + q < np;
            const int col = valid ? (ts.direct ? d.pc_col[k] : scol[k - kc]) : 0;
            const uint32_t ol = valid ? (ts.direct ? d.pc_ol[k] : sol[k - kc]) : 0u;
            const int len = (int)(ol & 63u);
            const int64_t eb = rb + (int64_t)(ol >> 6);
#pragma unroll
            for (int u = 0; u < PP; ++u) {
              const int j = gl + u * G;
              const bool in = j < len;
              const uint64_t b = (uint64_t)(eb + j) * Val<K>::B;
              xv[q * PP + u] = in ? __ldg(d.p32 + col + j) : 0.f;
              av[q * PP + u] = !in ? 0.f : Val<K>::dec(ts.direct ? gv + b : st + StageLayout::kVal + (b - ts.v.lo));
            }
          }
#pragma unroll
          for (int u = 0; u < NP * PP; ++u) acc[u & 3] = fmaf(av[u], xv[u], acc[u & 3]);
        }
        float a = (acc[0] + acc[1]) + (acc[2] + acc[3]);
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

static int staged_grid(const Dev& d) {
  const int64_t sm = d.sm_count > 0 ? d.sm_count : 148;
  return (int)std::max<int64_t>(1, std::min<int64_t>(d.ntiles, sm));
}

template <int K>
static void launch_staged_k(const Dev& d, int mode, cudaStream_t st) {
  const int grid = staged_grid(d);
  const size_t smem = (size_t)kStages * kStageAlloc;
  if (mode == 0) k_op_rows_staged<K, 0><<<grid, kStagedThreads, smem, st>>>(d);
  else k_op_rows_staged<K, 1><<<grid, kStagedThreads, smem, st>>>(d);
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
#define IPMK_SET_STAGED(K) \
  set((const void*)k_op_rows_staged<K, 0>); set((const void*)k_op_rows_staged<K, 1>);
  IPMK_SET_STAGED(ST_F64)
  IPMK_SET_STAGED(ST_F32)
  IPMK_SET_STAGED(ST_BF16)
  IPMK_SET_STAGED(ST_FP8)
#undef IPMK_SET_STAGED
  return e;
}

}  // namespace ipmk
