// Host-side preparation of a QP's matrices (multi-threaded; results identical to the
// sequential definitions).
#include "ingest.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

namespace ipmk {

int host_threads() {
  const unsigned hc = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(hc ? hc : 1u, 64u));
}

void parallel_ranges(int64_t n, int parts, const std::function<void(int, int64_t, int64_t)>& fn) {
  parts = (int)std::max<int64_t>(1, std::min<int64_t>(parts, n));
  if (parts == 1) {
    fn(0, 0, n);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(parts);
  for (int t = 0; t < parts; ++t) {
    const int64_t b = n * t / parts, e = n * (t + 1) / parts;
    th.emplace_back([&fn, t, b, e]() { fn(t, b, e); });
  }
  for (auto& x : th) x.join();
}

void par_copy(void* dst, const void* src, size_t nbytes) {
  if (nbytes == 0) return;
  const int T = nbytes < (size_t)(8 << 20) ? 1 : host_threads();
  parallel_ranges((int64_t)nbytes, T, [&](int, int64_t b, int64_t e) {
    std::memcpy(static_cast<char*>(dst) + b, static_cast<const char*>(src) + b, (size_t)(e - b));
  });
}

int check_csr_entries(int64_t nnz, const int32_t* idx, const double* val, int64_t ncols) {
  // each thread finds the first bad entry of its range; the answer is the code of the first
  // bad entry overall, as the sequential scan would report it
  const int T = nnz < (1 << 20) ? 1 : host_threads();
  std::vector<int64_t> first((size_t)T, -1);
  std::vector<int> code((size_t)T, 0);
  parallel_ranges(nnz, T, [&](int t, int64_t b, int64_t e) {
    for (int64_t k = b; k < e; ++k) {
      if (idx[k] < 0 || idx[k] >= ncols) { first[t] = k; code[t] = 1; break; }
      if (!std::isfinite(val[k])) { first[t] = k; code[t] = 2; break; }
    }
  });
  for (int t = 0; t < T; ++t)   // ranges are in order: the first thread with a bad entry wins
    if (first[t] >= 0) return code[t];
  return 0;
}

void transpose_csr(int64_t nrows, int64_t ncols, const int64_t* rp, const int32_t* ri, const double* rv,
                   int64_t* tp, int32_t* ti, double* tv) {
  const int64_t nnz = rp[nrows];
  // threads over row blocks of equal entry counts; the per-thread column counts must fit
  int T = nnz < (1 << 20) ? 1 : host_threads();
  T = (int)std::max<int64_t>(1, std::min<int64_t>(T, (int64_t)(256 << 20) / (8 * std::max<int64_t>(ncols, 1))));
  std::vector<int64_t> rb(T + 1);
  for (int t = 0; t <= T; ++t) {
    const int64_t target = nnz * t / T;
    rb[t] = std::lower_bound(rp, rp + nrows + 1, target) - rp;
  }
  rb[0] = 0;
  rb[T] = nrows;
  std::vector<int64_t> cnt((size_t)T * (size_t)ncols, 0);
  parallel_ranges(T, T, [&](int, int64_t tb, int64_t) {
    const int t = (int)tb;
    int64_t* c = cnt.data() + (size_t)t * ncols;
    for (int64_t e = rp[rb[t]]; e < rp[rb[t + 1]]; ++e) c[ri[e]]++;
  });
  // per column: exclusive offsets of the thread blocks, then column totals
  std::vector<int64_t> tot(ncols);
  parallel_ranges(ncols, T, [&](int, int64_t jb, int64_t je) {
    for (int64_t j = jb; j < je; ++j) {
      int64_t run = 0;
      for (int t = 0; t < T; ++t) {
        int64_t& c = cnt[(size_t)t * ncols + j];
        const int64_t v = c;
        c = run;
        run += v;
      }
      tot[j] = run;
    }
  });
  tp[0] = 0;
  for (int64_t j = 0; j < ncols; ++j) tp[j + 1] = tp[j] + tot[j];
  parallel_ranges(T, T, [&](int, int64_t tb, int64_t) {
    const int t = (int)tb;
    int64_t* cur = cnt.data() + (size_t)t * ncols;
    for (int64_t r = rb[t]; r < rb[t + 1]; ++r)
      for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
        const int32_t j = ri[e];
        const int64_t pos = tp[j] + cur[j]++;
        ti[pos] = (int32_t)r;
        tv[pos] = rv[e];
      }
  });
}

void filter_rows(int64_t ncols, const int64_t* tp, const int32_t* ti, const double* tv, const unsigned char* keep,
                 int64_t* op, int32_t* oi, double* ov) {
  const int T = tp[ncols] < (1 << 20) ? 1 : host_threads();
  if (!oi) {
    std::vector<int64_t> c(ncols);
    parallel_ranges(ncols, T, [&](int, int64_t jb, int64_t je) {
      for (int64_t j = jb; j < je; ++j) {
        int64_t k = 0;
        for (int64_t e = tp[j]; e < tp[j + 1]; ++e) k += keep[ti[e]] ? 1 : 0;
        c[j] = k;
      }
    });
    op[0] = 0;
    for (int64_t j = 0; j < ncols; ++j) op[j + 1] = op[j] + c[j];
    return;
  }
  parallel_ranges(ncols, T, [&](int, int64_t jb, int64_t je) {
    for (int64_t j = jb; j < je; ++j) {
      int64_t o = op[j];
      for (int64_t e = tp[j]; e < tp[j + 1]; ++e)
        if (keep[ti[e]]) {
          oi[o] = ti[e];
          ov[o] = tv[e];
          ++o;
        }
    }
  });
}

void order_rows_by_length(int64_t nrows, const int64_t* rp, int window, int32_t* perm) {
  if (nrows <= 0) return;
  const int64_t nw = (nrows + window - 1) / window;
  const int T = nrows < (1 << 16) ? 1 : host_threads();
  parallel_ranges(nw, T, [&](int, int64_t wb, int64_t we) {
    std::vector<std::pair<int64_t, int32_t>> key;    // (-length, row): ascending = longest first, stable
    for (int64_t w = wb; w < we; ++w) {
      const int64_t r0 = w * window, r1 = std::min<int64_t>(nrows, r0 + window);
      key.clear();
      for (int64_t r = r0; r < r1; ++r) key.emplace_back(-(rp[r + 1] - rp[r]), (int32_t)r);
      std::sort(key.begin(), key.end());
      for (int64_t r = r0; r < r1; ++r) perm[r] = key[r - r0].second;
    }
  });
}

}  // namespace ipmk
