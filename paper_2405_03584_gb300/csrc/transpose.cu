// Device-side preparation of R^T and A^T at ipm_set_qp.
//
// R (CSR) is uploaded as given; its entries are checked, counted per column, scattered into
// the columns of R^T with atomic cursors, and each column is then sorted by row index, which
// gives the unique order of the sequential stable counting sort (rows increase within a
// column; a row holds a column at most once).  A^T is the ordered subset of R^T on
// constraint rows (one warp per column, ballot-ordered copy).  The result is bit-for-bit
// the host transpose's (ingest.cu), which stays as the fallback for columns longer than the
// in-block sort holds.
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "transpose.h"

namespace ipmk {
namespace {

constexpr int kSortMax = 4096;   // longest column sorted in shared memory
constexpr int kTB = 256;

__global__ void k_tr_check_count(const int32_t* __restrict__ ri, const double* __restrict__ rv, int64_t nnz,
                                 int64_t n, int* __restrict__ cnt, int* __restrict__ flag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = ri[e];
    if (j < 0 || j >= n) {
      atomicOr(flag, 1);
      continue;
    }
    if (!isfinite(rv[e])) atomicOr(flag, 2);
    atomicAdd(cnt + j, 1);
  }
}

// Exclusive scan of n counts into ptr[0..n] (one block: a serial chunk per thread, then a
// block scan of the chunk totals); the largest count into *maxlen.
__global__ void k_tr_scan(const int* __restrict__ cnt, int64_t n, int64_t* __restrict__ ptr, int* __restrict__ maxlen) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int64_t per = (n + T - 1) / T;
  const int64_t b = t * per, e = b + per < n ? b + per : n;
  int64_t s = 0;
  int mx = 0;
  for (int64_t j = b; j < e; ++j) {
    s += cnt[j];
    mx = max(mx, cnt[j]);
  }
  part[t] = s;
  atomicMax(maxlen, mx);
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int k = 0; k < T; ++k) {
      const int64_t v = part[k];
      part[k] = run;
      run += v;
    }
    ptr[n] = run;
  }
  __syncthreads();
  int64_t run = part[t];
  for (int64_t j = b; j < e; ++j) {
    ptr[j] = run;
    run += cnt[j];
  }
}

// One warp per row: entry (r, j, v) goes to column j at an atomic cursor.
__global__ void k_tr_fill(const int64_t* __restrict__ rp, const int32_t* __restrict__ ri, const double* __restrict__ rv,
                          int64_t nR, const int64_t* __restrict__ tp, int* __restrict__ cur, int32_t* __restrict__ ti,
                          double* __restrict__ tv) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < nR;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    for (int64_t e = rp[r] + lane; e < rp[r + 1]; e += 32) {
      const int32_t j = ri[e];
      const int64_t pos = tp[j] + atomicAdd(cur + j, 1);
      ti[pos] = (int32_t)r;
      tv[pos] = rv[e];
    }
  }
}

// One block per column: bitonic sort of (row, value) by row in shared memory.
__global__ void k_tr_sort(const int64_t* __restrict__ tp, int64_t n, int32_t* __restrict__ ti, double* __restrict__ tv) {
  __shared__ int key[kSortMax];
  __shared__ double val[kSortMax];
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const int64_t b = tp[j];
    const int L = (int)(tp[j + 1] - b);
    if (L <= 1) continue;
    int P = 1;
    while (P < L) P <<= 1;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
      key[k] = k < L ? ti[b + k] : INT_MAX;
      val[k] = k < L ? tv[b + k] : 0.0;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int k = threadIdx.x; k < P; k += blockDim.x) {
          const int o = k ^ stride;
          if (o > k) {
            const bool up = (k & size) == 0;
            if ((key[k] > key[o]) == up) {
              const int tk = key[k]; key[k] = key[o]; key[o] = tk;
              const double tw = val[k]; val[k] = val[o]; val[o] = tw;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
      ti[b + k] = key[k];
      tv[b + k] = val[k];
    }
    __syncthreads();
  }
}

__global__ void k_tr_mark(const int32_t* __restrict__ arow, int64_t m, unsigned char* __restrict__ is_con) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    is_con[arow[k]] = 1;
}

// A^T counts: entries of each column of R^T on constraint rows (one warp per column).
__global__ void k_tr_at_count(const int64_t* __restrict__ tp, const int32_t* __restrict__ ti, int64_t n,
                              const unsigned char* __restrict__ is_con, int* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  for (int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; j < n;
       j += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    int c = 0;
    for (int64_t e = tp[j] + lane; e < tp[j + 1]; e += 32) c += is_con[ti[e]];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[j] = c;
  }
}

// A^T fill in R^T's order (one warp per column, ballot-ordered).
__global__ void k_tr_at_fill(const int64_t* __restrict__ tp, const int32_t* __restrict__ ti, const double* __restrict__ tv,
                             int64_t n, const unsigned char* __restrict__ is_con, const int64_t* __restrict__ atp,
                             int32_t* __restrict__ ati, double* __restrict__ atv) {
  const int lane = threadIdx.x & 31;
  for (int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; j < n;
       j += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    int64_t out = atp[j];
    for (int64_t e0 = tp[j]; e0 < tp[j + 1]; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool keep = e < tp[j + 1] && is_con[ti[e]];
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int64_t pos = out + __popc(bal & ((1u << lane) - 1u));
        ati[pos] = ti[e];
        atv[pos] = tv[e];
      }
      out += __popc(bal);
    }
  }
}

int blocks(int64_t items, int per, int cap) {
  int64_t b = (items + per - 1) / per;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

}  // namespace

size_t device_transpose_scratch(int64_t n, int64_t nR) {
  return 3 * 256 + sizeof(int) * 2 * (size_t)(n + 1) + (size_t)nR + 64;
}

int device_transpose(const int64_t* rp, const int32_t* ri, const double* rv, int64_t nR, int64_t n, int64_t nnz,
                     const int32_t* arow, int64_t m, int64_t* tp, int32_t* ti, double* tv, int64_t* atp, int32_t* ati,
                     double* atv, void* scratch, int sm_count, cudaStream_t st, cudaError_t* err) {
  char* p = static_cast<char*>(scratch);
  int* cnt = reinterpret_cast<int*>(p);
  int* cur = cnt + (n + 1);
  unsigned char* is_con = reinterpret_cast<unsigned char*>(cur + (n + 1));
  int* flags = reinterpret_cast<int*>(((uintptr_t)(is_con + nR) + 255) & ~(uintptr_t)255);   // flag, maxlen
  const int cap = 8 * (sm_count > 0 ? sm_count : 148);
  int host_flags[2] = {0, 0};
  *err = cudaSuccess;
  auto chk = [&](cudaError_t e) {
    if (e != cudaSuccess && *err == cudaSuccess) *err = e;
    return e == cudaSuccess;
  };
  if (!chk(cudaMemsetAsync(cnt, 0, sizeof(int) * 2 * (size_t)(n + 1), st))) return -1;
  if (!chk(cudaMemsetAsync(flags, 0, 2 * sizeof(int), st))) return -1;
  if (nnz) k_tr_check_count<<<blocks(nnz, kTB, cap), kTB, 0, st>>>(ri, rv, nnz, n, cnt, flags);
  k_tr_scan<<<1, 1024, 0, st>>>(cnt, n, tp, flags + 1);
  if (!chk(cudaGetLastError())) return -1;
  if (!chk(cudaMemcpyAsync(host_flags, flags, sizeof(host_flags), cudaMemcpyDeviceToHost, st))) return -1;
  if (!chk(cudaStreamSynchronize(st))) return -1;
  if (host_flags[0] & 1) return 1;
  if (host_flags[0] & 2) return 2;
  if (host_flags[1] > kSortMax) return 3;
  if (nnz) {
    k_tr_fill<<<blocks(nR * 32, kTB, cap), kTB, 0, st>>>(rp, ri, rv, nR, tp, cur, ti, tv);
    k_tr_sort<<<blocks(n, 1, cap), kTB, 0, st>>>(tp, n, ti, tv);
  }
  // A^T over the constraint rows
  if (!chk(cudaMemsetAsync(is_con, 0, (size_t)(nR > 0 ? nR : 1), st))) return -1;
  if (m) k_tr_mark<<<blocks(m, kTB, cap), kTB, 0, st>>>(arow, m, is_con);
  k_tr_at_count<<<blocks(n * 32, kTB, cap), kTB, 0, st>>>(tp, ti, n, is_con, cnt);
  k_tr_scan<<<1, 1024, 0, st>>>(cnt, n, atp, flags + 1);
  k_tr_at_fill<<<blocks(n * 32, kTB, cap), kTB, 0, st>>>(tp, ti, tv, n, is_con, atp, ati, atv);
  if (!chk(cudaGetLastError())) return -1;
  return 0;
}

}  // namespace ipmk
