"""The host-side ingest routines (csrc/ingest.cu: the transpose fallback of ipm_set_qp and
options.ingest_host, the row order of the rows pass) on the CPU: compiled with the host compiler into a small driver and
compared with scipy's transpose, on a matrix large enough for the multi-threaded paths.
The results must be those of the sequential definitions, whatever the thread count."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2405_03584_gb300 import workloads as W

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2405_03584_gb300", "csrc")

DRIVER = r"""
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>
#include "ingest.h"

template <typename T> static std::vector<T> rd(const std::string& p, size_t n) {
  std::vector<T> v(n);
  FILE* f = std::fopen(p.c_str(), "rb");
  if (!f || std::fread(v.data(), sizeof(T), n, f) != n) std::exit(3);
  std::fclose(f);
  return v;
}
template <typename T> static void wr(const std::string& p, const std::vector<T>& v) {
  FILE* f = std::fopen(p.c_str(), "wb");
  if (!f || std::fwrite(v.data(), sizeof(T), v.size(), f) != v.size()) std::exit(4);
  std::fclose(f);
}
int main(int argc, char** argv) {
  const std::string d = argv[1];
  auto meta = rd<int64_t>(d + "/meta", 3);
  const int64_t nr = meta[0], nc = meta[1], nnz = meta[2];
  auto rp = rd<int64_t>(d + "/rp", nr + 1);
  auto ri = rd<int32_t>(d + "/ri", nnz);
  auto rv = rd<double>(d + "/rv", nnz);
  auto keep = rd<unsigned char>(d + "/keep", nr);
  std::vector<int64_t> tp(nc + 1), op(nc + 1);
  std::vector<int32_t> ti(nnz);
  std::vector<double> tv(nnz);
  ipmk::transpose_csr(nr, nc, rp.data(), ri.data(), rv.data(), tp.data(), ti.data(), tv.data());
  ipmk::filter_rows(nc, tp.data(), ti.data(), tv.data(), keep.data(), op.data(), nullptr, nullptr);
  std::vector<int32_t> oi(op[nc]);
  std::vector<double> ov(op[nc]);
  ipmk::filter_rows(nc, tp.data(), ti.data(), tv.data(), keep.data(), op.data(), oi.data(), ov.data());
  std::vector<int64_t> codes(3);
  codes[0] = ipmk::check_csr_entries(nnz, ri.data(), rv.data(), nc);
  auto bad_i = ri;
  bad_i[nnz / 2] = (int32_t)nc;
  codes[1] = ipmk::check_csr_entries(nnz, bad_i.data(), rv.data(), nc);
  auto bad_v = rv;
  bad_v[nnz - 1] = NAN;
  codes[2] = ipmk::check_csr_entries(nnz, ri.data(), bad_v.data(), nc);
  // a NaN early and a bad index late (different thread ranges), and the other way round: the
  // code of the first bad entry, whatever thread finishes first
  auto both_i = ri;
  auto both_v = rv;
  both_v[1] = NAN;
  both_i[nnz - 2] = -1;
  codes.push_back(ipmk::check_csr_entries(nnz, both_i.data(), both_v.data(), nc));
  both_v[1] = rv[1];
  both_v[nnz - 2] = NAN;
  both_i[nnz - 2] = ri[nnz - 2];
  both_i[2] = (int32_t)nc + 7;
  codes.push_back(ipmk::check_csr_entries(nnz, both_i.data(), both_v.data(), nc));
  std::vector<double> cp(nnz);
  ipmk::par_copy(cp.data(), rv.data(), sizeof(double) * nnz);
  codes.push_back(cp == rv ? 1 : 0);
  std::vector<int32_t> perm(nr);
  ipmk::order_rows_by_length(nr, rp.data(), 1024, perm.data());
  wr(d + "/perm", perm);
  wr(d + "/tp", tp); wr(d + "/ti", ti); wr(d + "/tv", tv);
  wr(d + "/op", op); wr(d + "/oi", oi); wr(d + "/ov", ov); wr(d + "/codes", codes);
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("ingest")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I" + CSRC, str(src), "-x", "c++",
                        os.path.join(CSRC, "ingest.cu"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe)


@pytest.mark.parametrize("n,density,seed", [(2000, 0.1, 3), (11, 0.3, 4)])
def test_host_transpose_filter_and_checks(driver, tmp_path, n, density, seed):
    """n = 2000 at 10% density gives 8000 x 2000 with about 1.6e6 entries (above the 2^20
    threshold of the threaded paths); n = 11 a tiny ragged case."""
    p = W.rt_qp(n=n, density=density, seed=seed)
    if n > 100:
        assert p["D_indptr"][-1] > (1 << 20)
    nr, nc = p["V"], p["n"]
    rp, ri, rv = p["D_indptr"].astype(np.int64), p["D_indices"].astype(np.int32), p["D_data"].astype(np.float64)
    keep = (np.random.default_rng(seed).random(nr) < 0.3).astype(np.uint8)
    nnz = int(rp[-1])
    np.array([nr, nc, nnz], np.int64).tofile(tmp_path / "meta")
    rp.tofile(tmp_path / "rp")
    ri.tofile(tmp_path / "ri")
    rv.tofile(tmp_path / "rv")
    keep.tofile(tmp_path / "keep")
    r = subprocess.run([driver, str(tmp_path)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    ld = lambda name, dt: np.fromfile(tmp_path / name, dtype=dt)
    T = sp.csr_matrix((rv, ri, rp), shape=(nr, nc)).T.tocsr()
    T.sort_indices()
    assert np.array_equal(ld("tp", np.int64), T.indptr)
    assert np.array_equal(ld("ti", np.int32), T.indices)
    assert np.array_equal(ld("tv", np.float64), T.data)
    mask = keep[T.indices].astype(bool)
    rows = np.repeat(np.arange(nc), np.diff(T.indptr))
    op = np.concatenate([[0], np.cumsum(np.bincount(rows[mask], minlength=nc))])
    assert np.array_equal(ld("op", np.int64), op)
    assert np.array_equal(ld("oi", np.int32), T.indices[mask])
    assert np.array_equal(ld("ov", np.float64), T.data[mask])
    assert list(ld("codes", np.int64)) == [0, 1, 2, 2, 1, 1]
    # rows-pass order: windows of 1024 rows, longest first, ties in row order
    lens = np.diff(rp)
    want = np.concatenate([w0 + np.argsort(-lens[w0:w0 + 1024], kind="stable") for w0 in range(0, nr, 1024)])
    assert np.array_equal(ld("perm", np.int32), want)
