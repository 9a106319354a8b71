// Device-side preparation of R^T and A^T at ipm_set_qp (transpose.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace ipmk {

// Bytes of device scratch device_transpose needs for n columns and nR rows.
size_t device_transpose_scratch(int64_t n, int64_t nR);

// R (rp, ri, rv: nR rows, nnz entries, columns in [0, n) expected) -> R^T (tp: n + 1, ti, tv)
// with rows increasing within each column, and A^T (atp: n + 1, ati, atv: the entries of R^T
// on the m constraint rows arow, same order).  Device pointers; synchronises the stream once
// (after the checks).  Returns 0 on success, 1 if a column index is out of range, 2 if a
// value is not finite, 3 if a column is longer than the device sort holds (nothing written:
// use the host transpose), -1 on a CUDA error (*err set).
int device_transpose(const int64_t* rp, const int32_t* ri, const double* rv, int64_t nR, int64_t n, int64_t nnz,
                     const int32_t* arow, int64_t m, int64_t* tp, int32_t* ti, double* tv, int64_t* atp, int32_t* ati,
                     double* atv, void* scratch, int sm_count, cudaStream_t st, cudaError_t* err);

}  // namespace ipmk
