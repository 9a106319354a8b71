// Dense pieces of the preconditioners (sm_103a, float64):
//   * k_gram_K   : K = Hs + R^T diag(omega) R + diag(h0 + sigma) as a dense n x n matrix
//                  (the DENSE preconditioner: one diagonal block covering all variables);
//   * k_chol     : in-place Cholesky factor (lower) with pivot flooring, one block;
//   * k_mirror   : copies L into the upper triangle so both sweeps of the inverse read rows;
//   * k_inv      : explicit inverse from the factor, columns spread over blocks.
// The explicit inverse turns every preconditioner apply inside PCG into a parallel matvec;
// the factorisation runs once per IPM iteration.
#include <algorithm>
#include <cmath>

#include "state.h"

namespace ipmk {

// One block per row j of K.  Rows of R are summed in the fixed order of the stored
// transpose; the entries of one row of R have distinct columns, so threads never collide.
__global__ void k_gram_K(Dev d) {
  extern __shared__ double row[];
  const int64_t n = d.n;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) row[i] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) row[j] = d.h0[j] + d.sigma[j];
    __syncthreads();
    if (d.Hs_ptr) {
      for (int64_t e = d.Hs_ptr[j] + threadIdx.x; e < d.Hs_ptr[j + 1]; e += blockDim.x) row[d.Hs_idx[e]] += d.Hs_val[e];
      __syncthreads();
    }
    for (int64_t e = d.RT_ptr[j]; e < d.RT_ptr[j + 1]; ++e) {
      const int32_t i = d.RT_idx[e];
      const double f = d.RT_val[e] * d.omega[i];
      if (f != 0.0)
        for (int64_t t = d.R_ptr[i] + threadIdx.x; t < d.R_ptr[i + 1]; t += blockDim.x) row[d.R_idx[t]] += f * d.R_val[t];
      __syncthreads();
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) d.Kd[j * n + i] = row[i];
    __syncthreads();
  }
}

// Right-looking Cholesky of the leading nn x nn block of A (row-major, leading dimension ld),
// lower triangle overwritten by L.  A pivot below floor_rel * (original diagonal) is raised
// to that floor (a modified factor; still symmetric positive definite, which is all a
// preconditioner needs); the count of floored pivots goes to *nfloor.
// Shared memory: 2 * nn doubles (column cache and original diagonal).
__global__ void k_chol(double* A, int64_t ld, const int* nn_dev, int nn_fixed, double floor_rel, int* nfloor) {
  extern __shared__ double shm[];
  const int nn = nn_dev ? *nn_dev : nn_fixed;
  double* colk = shm;
  double* diag0 = shm + nn;
  for (int i = threadIdx.x; i < nn; i += blockDim.x) diag0[i] = A[(int64_t)i * ld + i];
  __shared__ double s_lkk;
  __shared__ int s_floor;
  if (threadIdx.x == 0) s_floor = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < nn; ++k) {
    if (threadIdx.x == 0) {
      double akk = A[(int64_t)k * ld + k];
      const double fl = floor_rel * fabs(diag0[k]) + 1e-300;
      if (!(akk > fl)) { akk = fl; s_floor += 1; }
      const double lkk = sqrt(akk);
      A[(int64_t)k * ld + k] = lkk;
      s_lkk = lkk;
    }
    __syncthreads();
    const double inv = 1.0 / s_lkk;
    for (int i = k + 1 + threadIdx.x; i < nn; i += blockDim.x) {
      const double v = A[(int64_t)i * ld + k] * inv;
      A[(int64_t)i * ld + k] = v;
      colk[i] = v;
    }
    __syncthreads();
    // trailing update of the lower triangle: A[i][j] -= L[i][k] L[j][k], k < j <= i
    for (int i = k + 1 + wid; i < nn; i += nw) {
      const double lik = colk[i];
      double* ai = A + (int64_t)i * ld;
      for (int j = k + 1 + lane; j <= i; j += 32) ai[j] = fma(-lik, colk[j], ai[j]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && nfloor) *nfloor = s_floor;
}

// Upper triangle <- L^T so that column p of L is row p of the upper part.
__global__ void k_mirror(double* A, int64_t ld, const int* nn_dev, int nn_fixed) {
  const int nn = nn_dev ? *nn_dev : nn_fixed;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)nn * nn; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t / nn, i = t % nn;
    if (i > p) A[p * ld + i] = A[i * ld + p];
  }
}

// Column c of A^{-1} = L^{-T} L^{-1} e_c: forward sweep reads row p of the upper part (= column
// p of L), backward sweep reads row q of L; both contiguous.  One block per column at a time.
__global__ void k_inv(const double* A, int64_t ld, const int* nn_dev, int nn_fixed, double* Ainv, int64_t ldi) {
  extern __shared__ double y[];
  const int nn = nn_dev ? *nn_dev : nn_fixed;
  for (int c = blockIdx.x; c < nn; c += gridDim.x) {
    for (int i = threadIdx.x; i < nn; i += blockDim.x) y[i] = (i == c) ? 1.0 : 0.0;
    __syncthreads();
    for (int p = c; p < nn; ++p) {
      const double yp = y[p] / A[(int64_t)p * ld + p];
      __syncthreads();
      if (threadIdx.x == 0) y[p] = yp;
      const double* up = A + (int64_t)p * ld;
      for (int i = p + 1 + threadIdx.x; i < nn; i += blockDim.x) y[i] = fma(-up[i], yp, y[i]);
      __syncthreads();
    }
    for (int q = nn - 1; q >= 0; --q) {
      const double xq = y[q] / A[(int64_t)q * ld + q];
      __syncthreads();
      if (threadIdx.x == 0) y[q] = xq;
      const double* lq = A + (int64_t)q * ld;
      for (int i = threadIdx.x; i < q; i += blockDim.x) y[i] = fma(-lq[i], xq, y[i]);
      __syncthreads();
    }
    for (int i = threadIdx.x; i < nn; i += blockDim.x) Ainv[(int64_t)i * ldi + c] = y[i];
    __syncthreads();
  }
}

cudaError_t launch_dense_build(const Dev& d, cudaStream_t st) {
  const int n = (int)d.n;
  const size_t rowbytes = sizeof(double) * (size_t)n;
  k_gram_K<<<(int)std::min<int64_t>(d.n, 4 * 152), 256, rowbytes, st>>>(d);
  k_chol<<<1, 1024, 2 * rowbytes, st>>>(d.Kd, d.n, nullptr, n, 1e-13, &d.sc->chol_fail);
  k_mirror<<<256, 256, 0, st>>>(d.Kd, d.n, nullptr, n);
  k_inv<<<(int)std::min<int64_t>(d.n, 4 * 152), 256, rowbytes, st>>>(d.Kd, d.n, nullptr, n, d.Kinv, d.n);
  return cudaGetLastError();
}

cudaError_t launch_stiff_factor(const Dev& d, cudaStream_t st) {
  const int cap = d.stiff_cap;
  const size_t rowbytes = sizeof(double) * (size_t)cap;
  const int* ns = &d.sc->n_stiff;
  k_chol<<<1, 1024, 2 * rowbytes, st>>>(d.G, cap, ns, 0, 1e-13, &d.sc->chol_fail);
  k_mirror<<<64, 256, 0, st>>>(d.G, cap, ns, 0);
  k_inv<<<std::min(cap, 4 * 152), 256, rowbytes, st>>>(d.G, cap, ns, 0, d.Ginv, cap);
  return cudaGetLastError();
}

}  // namespace ipmk
