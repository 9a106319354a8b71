// Host-side preparation of a QP's matrices at ipm_set_qp, multi-threaded.  Every routine
// gives exactly the result of its sequential definition (same order, same values), whatever
// the number of threads.
#pragma once
#include <cstdint>
#include <functional>

namespace ipmk {

// Worker threads used by the host preparation (hardware threads, at most 64).
int host_threads();

// Runs fn(t, begin, end) on [0, n) split into `parts` contiguous ranges, one thread each.
void parallel_ranges(int64_t n, int parts, const std::function<void(int, int64_t, int64_t)>& fn);

// Parallel memcpy of nbytes.
void par_copy(void* dst, const void* src, size_t nbytes);

// Checks every column index in [0, ncols) and every value finite.  Returns 0 if all are
// valid, 1 for an index out of range, 2 for a value that is not finite.
int check_csr_entries(int64_t nnz, const int32_t* idx, const double* val, int64_t ncols);

// Stable transpose of a CSR matrix (nrows x ncols): within each column the entries keep
// increasing row order (the sequential counting sort's order).  tp: ncols + 1 pointers.
void transpose_csr(int64_t nrows, int64_t ncols, const int64_t* rp, const int32_t* ri, const double* rv,
                   int64_t* tp, int32_t* ti, double* tv);

// The entries of a transposed CSR (tp, ti, tv over ncols columns) whose row index r has
// keep[r] != 0, in the same order: out pointers op (ncols + 1), then oi, ov sized op[ncols].
// Two calls: with oi == nullptr only op is filled.
void filter_rows(int64_t ncols, const int64_t* tp, const int32_t* ti, const double* tv, const unsigned char* keep,
                 int64_t* op, int32_t* oi, double* ov);

// Row order of the rows pass: windows of `window` consecutive rows, each ordered by row
// length, longest first, ties in row order (a stable sort).  perm: nrows entries.
void order_rows_by_length(int64_t nrows, const int64_t* rp, int window, int32_t* perm);

}  // namespace ipmk
