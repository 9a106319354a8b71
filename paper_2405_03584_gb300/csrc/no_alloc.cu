// Allocation-free apply of the condensed PCG operator, for callers that cannot allocate
// device memory: code running where cudaMalloc is off limits (inside an application that
// owns and budgets all device memory itself, a custom allocator that must not recurse into
// the CUDA allocator, or a framework hook that may not allocate).  The caller passes every
// input and output; the one intermediate vector (v = omega o (R p), one double per row of R)
// lives in a file-scope device array instead of an allocation.
//
// The array holds IPM_STATIC_SCRATCH_ROWS doubles (2 MiB) on every GPU that loads this
// library, until the process exits.  All calls share it and it keeps the last call's
// contents; every element a call reads was written earlier in the same call, so nothing has
// to start at zero.  Calls that overlap on the GPU (two streams, or two host threads) race on
// the array: serialise them.
#include <mutex>

#include "../../include/ipm.h"
#include "common.cuh"

namespace {

constexpr int64_t kStaticRows = IPM_STATIC_SCRATCH_ROWS;   // 2 MiB of doubles
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_v[kStaticRows];

// Device address of g_static_v per device, looked up once with that device current.
double* g_static_ptr[kMaxDevices] = {nullptr};
std::mutex g_static_mu;

// v_r = omega_r (R_r . p), one warp per row, into the static array.
__global__ void k_static_rows(int64_t nR, const int64_t* __restrict__ Rp, const int32_t* __restrict__ Ri,
                              const double* __restrict__ Rv, const double* __restrict__ omega,
                              const double* __restrict__ p, double* __restrict__ v) {
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < nR; r += nw) {
    const double t = ipmk::warp_row_dot<false>(Rp[r], Rp[r + 1], Ri, Rv, p);
    if ((threadIdx.x & 31) == 0) v[r] = omega[r] * t;
  }
}

// q_j = R^T_j . v + dg_j p_j, one warp per variable.
__global__ void k_static_cols(int64_t n, const int64_t* __restrict__ RTp, const int32_t* __restrict__ RTi,
                              const double* __restrict__ RTv, const double* __restrict__ v,
                              const double* __restrict__ dg, const double* __restrict__ p, double* __restrict__ q) {
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w0; j < n; j += nw) {
    const double acc = ipmk::warp_row_dot<false>(RTp[j], RTp[j + 1], RTi, RTv, v);
    if ((threadIdx.x & 31) == 0) q[j] = acc + dg[j] * p[j];
  }
}

// Looks up (once per device, under a lock, with that device current) the device address of
// the static array; the host-side symbol itself is not a device address.
int static_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return IPM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_v) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return IPM_ERR_CUDA;
    }
    g_static_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = g_static_ptr[dev];
  return IPM_OK;
}

}  // namespace

extern "C" int ipm_apply_operator_static(int64_t n, int64_t nR, const int64_t* R_indptr, const int32_t* R_indices,
                                         const double* R_data, const int64_t* RT_indptr, const int32_t* RT_indices,
                                         const double* RT_data, const double* omega, const double* dg,
                                         const double* p, double* q, void* stream) {
  // every pointer a launch below would dereference is checked before the size check, so a
  // NULL never reaches the device
  if (n < 1 || nR < 0 || !RT_indptr || !RT_indices || !RT_data || !dg || !p || !q) return IPM_ERR_ARG;
  if (nR > 0 && (!R_indptr || !R_indices || !R_data || !omega)) return IPM_ERR_ARG;
  if (nR > kStaticRows) return IPM_ERR_TOO_LARGE;
  double* v = nullptr;
  int rc = static_scratch(&v);
  if (rc != IPM_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = ipmk::kBlock, wpb = threads / 32;
  if (nR > 0) {
    const int64_t gb = (nR + wpb - 1) / wpb;
    k_static_rows<<<(int)(gb < 4096 ? gb : 4096), threads, 0, st>>>(nR, R_indptr, R_indices, R_data, omega, p, v);
  }
  const int64_t gb = (n + wpb - 1) / wpb;
  k_static_cols<<<(int)(gb < 4096 ? gb : 4096), threads, 0, st>>>(n, RT_indptr, RT_indices, RT_data, v, dg, p, q);
  if (cudaGetLastError() != cudaSuccess) return IPM_ERR_CUDA;
  return IPM_OK;
}
