// C ABI of the interior point library (declared in include/ipm.h): handle, problem ingest,
// device arena, the captured CUDA graph of a whole solve, asynchronous and batched launches.
//
// Control flow of ipm_solve: one CUDA graph per solve, all on the device.  Start point, then a
// conditional-while node over IPM iterations (Algorithm 1) whose body is: diagonal update ->
// preconditioner build -> right-hand side -> PCG as a nested conditional-while node (one trip
// per PCG iteration; the condition is set by the last kernel of the trip) -> direction
// recovery -> ratio test -> update -> residual summary -> mu test / stop rule (which sets the
// outer condition and appends a trace row).  The host launches the graph and waits once.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ipm.h"
#include "ingest.h"
#include "state.h"
#include "transpose.h"

using namespace ipmk;

namespace {

// Kernel nodes at each loop level of a captured graph (for launch accounting).
struct LoopCounts {
  int top = 0;       // outside every loop
  int ipm = 0;       // IPM-loop body, outside nested loops
  int pcg = 0;       // one PCG trip
  int refine = 0;    // refinement body, outside its PCG loop
  int fallback = 0;  // one trip of the FP64 fallback loop
  int ru = 0;        // reduced precision with residual replacement: one PCG loop per step
};

struct Graphs {
  cudaGraphExec_t solve[2] = {nullptr, nullptr};   // whole solve: cold, warm
  cudaGraph_t solve_g[2] = {nullptr, nullptr};     // its un-instantiated graph (batch capture)
  cudaGraphExec_t dir = nullptr;                   // Newton direction only (PCG + recovery)
  LoopCounts solve_c[2], dir_c;
};

// Kernel nodes of a graph (not descending into child graphs).
int count_kernel_nodes(cudaGraph_t g) {
  size_t nn = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess) return 0;
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn && cudaGraphGetNodes(g, nodes.data(), &nn) != cudaSuccess) return 0;
  int k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

// Read-only device copy of a QP's matrices.  Handles that share a QP hold a reference; the
// memory is freed with the last one.
struct MatStore {
  void* ptr = nullptr;
  void* aux = nullptr;              // runs of R's rows (sized only once R is on the device)
  void* blk = nullptr;              // segments of the block-Jacobi preconditioner
  void* gap = nullptr;              // gap layout of R^T (reduced-precision column pass)
  size_t bytes = 0;
  int device = 0;
  int storage = 0;
  std::vector<int64_t> sc_prefix;   // entries of the k longest constraint rows, k = 0..min(m, 1024)
  ~MatStore() {
    if (ptr) {
      int cur = 0;
      cudaGetDevice(&cur);
      cudaSetDevice(device);
      cudaFree(ptr);
      if (aux) cudaFree(aux);
      if (blk) cudaFree(blk);
      if (gap) cudaFree(gap);
      cudaSetDevice(cur);
    }
  }
};

}  // namespace

struct ipm_handle {
  ipm_options opt;
  int device = 0;
  cudaStream_t st = nullptr, st2 = nullptr, st3 = nullptr, st4 = nullptr;
  cudaEvent_t ev = nullptr;
  void* arena = nullptr;             // per-handle state: iterate, PCG and preconditioner work
  size_t arena_bytes = 0;
  std::shared_ptr<MatStore> mat;    // matrices (R, R^T, H block, reduced copies); shared by ipm_share_qp
  Dev d{};
  Geo g{};
  Scal* hs = nullptr;               // pinned host copy of the device scalars
  bool loaded = false, have_iterate = false;
  int precond = PC_JACOBI_LR;
  Graphs graphs[kPrecondKinds];
  std::string err;
  ipm_info info{};
  double cnorm = 0, bnorm = 0;
  int ncomp = 0;
  int64_t sc_cap = 0;
  int64_t fr = 0;                   // rows of the factor F (the first rows of R)
  // two-sided rows (ipm_qp.bl): stacked = the stored rows differ from the caller's; then
  // row_of gives the caller's row of every stored row, upper sides first (stored rows
  // [0, rows_up)), then lower sides
  bool stacked = false;
  int64_t m_user = 0, rows_up = 0;
  std::vector<int32_t> row_of;
  std::vector<double> trace;        // IPM_TRACE_COLS doubles per IPM iteration of the last solve
  double* htrace = nullptr;         // pinned: trace rows copied back after a solve
  int trace_cap = 0;
  int pending = 0;                  // an asynchronous solve was launched and not yet waited for
  // Bumped whenever the buffers or kernel parameters that a captured solve graph holds change
  // (arena freed, QP reloaded or shared, low-rank column count changed); a batch records it
  // per member at ipm_batch_create and refuses to launch on a mismatch.
  uint64_t gen = 0;
  int pending_pc = 0, pending_warm = 0;
  std::chrono::steady_clock::time_point t_launch;
};

namespace {

int fail(ipm_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

#define CUDA_TRY(h, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail((h), IPM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Copies n elements from host or device memory into a host vector.
template <typename T>
int fetch(ipm_handle* h, const T* src, int64_t n, int mem, std::vector<T>& out) {
  out.resize((size_t)std::max<int64_t>(n, 0));
  if (n <= 0) return IPM_OK;
  if (!src) return fail(h, IPM_ERR_ARG, "missing array");
  if (mem == IPM_MEM_DEVICE) {
    CUDA_TRY(h, cudaMemcpy(out.data(), src, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(out.data(), src, sizeof(T) * (size_t)n);
  }
  return IPM_OK;
}

// Copies n elements from host or device memory into dst (host).
template <typename T>
int fetch_into(ipm_handle* h, const T* src, int64_t n, int mem, T* dst) {
  if (n <= 0) return IPM_OK;
  if (!src) return fail(h, IPM_ERR_ARG, "missing array");
  if (mem == IPM_MEM_DEVICE) {
    CUDA_TRY(h, cudaMemcpy(dst, src, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost));
  } else {
    par_copy(dst, src, sizeof(T) * (size_t)n);
  }
  return IPM_OK;
}

void destroy_graphs(ipm_handle* h) {
  h->gen++;
  for (auto& g : h->graphs) {
    for (int w = 0; w < 2; ++w) {
      if (g.solve[w]) cudaGraphExecDestroy(g.solve[w]);
      if (g.solve_g[w]) cudaGraphDestroy(g.solve_g[w]);
      g.solve[w] = nullptr;
      g.solve_g[w] = nullptr;
    }
    if (g.dir) cudaGraphExecDestroy(g.dir);
    g.dir = nullptr;
  }
}

void free_arena(ipm_handle* h) {
  destroy_graphs(h);
  if (h->htrace) cudaFreeHost(h->htrace);
  h->htrace = nullptr;
  h->trace_cap = 0;
  if (h->arena) cudaFree(h->arena);
  h->arena = nullptr;
  h->arena_bytes = 0;
  h->mat.reset();
  h->loaded = h->have_iterate = false;
  h->d = Dev{};
}

// Bump allocator over one device allocation.
struct Carver {
  char* base;
  size_t off = 0;
  bool count_only;
  explicit Carver(char* b) : base(b), count_only(b == nullptr) {}
  template <typename T>
  T* take(int64_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = count_only ? nullptr : reinterpret_cast<T*>(base + off);
    off += sizeof(T) * (size_t)std::max<int64_t>(n, 1);
    return p;
  }
};

struct HostQP {
  int64_t n = 0, m = 0, nR = 0, fr = 0;
  std::vector<int64_t> Rp, RTp, ATp, Hp;
  std::vector<int32_t> Ri, RTi, ATi, Hi, arow;
  std::vector<double> Rv, RTv, ATv, Hv, wR, h0, c, b, l, u;
  int64_t ucols = 0;
  std::vector<double> U, uw;        // low-rank Hessian term: n x ucols (row-major), ucols weights
  std::vector<unsigned char> fl, fu;
};

// Matrix part of the device layout (shared between handles that share a QP).
void carve_matrix(Carver& cv, Dev& d, int64_t n, int64_t m, int64_t nR, int64_t nnzR, int64_t nnzA, int64_t nnzHs,
                  int storage, bool df) {
  d.R_ptr = cv.take<int64_t>(nR + 1); d.R_idx = cv.take<int32_t>(nnzR); d.R_val = cv.take<double>(nnzR);
  d.RT_ptr = cv.take<int64_t>(n + 1); d.RT_idx = cv.take<int32_t>(nnzR); d.RT_val = cv.take<double>(nnzR);
  d.AT_ptr = cv.take<int64_t>(n + 1); d.AT_idx = cv.take<int32_t>(nnzA); d.AT_val = cv.take<double>(nnzA);
  if (nnzHs) {
    d.Hs_ptr = cv.take<int64_t>(n + 1); d.Hs_idx = cv.take<int32_t>(nnzHs); d.Hs_val = cv.take<double>(nnzHs);
  } else {
    d.Hs_ptr = nullptr; d.Hs_idx = nullptr; d.Hs_val = nullptr;
  }
  d.arow = cv.take<int32_t>(m);
  d.rperm = cv.take<int32_t>(nR);
  if (storage != ST_F64) {
    const size_t vb = storage == ST_F32 ? 4 : (storage == ST_BF16 ? 2 : 1);
    d.Rq = cv.take<unsigned char>((int64_t)vb * nnzR);
    d.RTq = cv.take<unsigned char>((int64_t)vb * nnzR);
    d.scaleR = cv.take<float>(nR);
  } else {
    d.Rq = d.RTq = nullptr;
    d.scaleR = nullptr;
  }
  if (df) {
    d.R_df = cv.take<float2>(nnzR);
    d.RT_df = cv.take<float2>(nnzR);
  } else {
    d.R_df = d.RT_df = nullptr;
  }
}

// Per-handle part: problem vectors (costs may change per handle), iterate and work space.
void carve_state(Carver& cv, Dev& d, int64_t n, int64_t m, int64_t nR, int stiff_cap, int64_t sc_cap, bool dense,
                 int storage, int trace_cap, bool df, int64_t nblk) {
  d.wR = cv.take<double>(nR); d.h0 = cv.take<double>(n); d.c = cv.take<double>(n); d.b = cv.take<double>(m);
  d.l = cv.take<double>(n); d.u = cv.take<double>(n);
  d.fl = cv.take<unsigned char>(n); d.fu = cv.take<unsigned char>(n);
  d.diagH = cv.take<double>(n);
  d.x = cv.take<double>(n); d.s = cv.take<double>(m); d.y = cv.take<double>(m);
  d.zl = cv.take<double>(n); d.zu = cv.take<double>(n);
  d.theta = cv.take<double>(m); d.sigma = cv.take<double>(n); d.omega = cv.take<double>(nR);
  d.M0 = cv.take<double>(n); d.Minv = cv.take<double>(n + m); d.thR = cv.take<double>(nR);
  d.rd = cv.take<double>(n); d.rp = cv.take<double>(m); d.Hx = cv.take<double>(n); d.Aty = cv.take<double>(n);
  d.tR = cv.take<double>(nR); d.vR = cv.take<double>(nR); d.vR2 = cv.take<double>(nR);
  // PCG vectors hold n + m entries: the doubly augmented system appends the multipliers
  d.dx = cv.take<double>(n + m); d.r = cv.take<double>(n + m); d.z = cv.take<double>(n + m);
  d.p = cv.take<double>(n + m); d.q = cv.take<double>(n + m); d.rhs = cv.take<double>(n + m);
  d.ds = cv.take<double>(m); d.dy = cv.take<double>(m); d.dzl = cv.take<double>(n); d.dzu = cv.take<double>(n);
  d.ratio = cv.take<double>(m); d.slotR = cv.take<int32_t>(nR); d.stiff_k = cv.take<int32_t>(stiff_cap);
  d.rowk = cv.take<int32_t>(nR);
  d.sc_cnt = cv.take<int32_t>(n); d.sc_ptr = cv.take<int64_t>(n + 1);
  d.sc_slot = cv.take<int32_t>(sc_cap); d.sc_val = cv.take<double>(sc_cap); d.sc_cap = sc_cap;
  d.G = cv.take<double>((int64_t)stiff_cap * stiff_cap); d.Ginv = cv.take<double>((int64_t)stiff_cap * stiff_cap);
  d.us = cv.take<double>(stiff_cap); d.ts = cv.take<double>(stiff_cap); d.stiff_cap = stiff_cap;
  d.us2 = cv.take<double>(stiff_cap);
  d.hist = cv.take<unsigned int>(kHistBins);
  d.Kd = dense ? cv.take<float2>(n * n) : nullptr;
  // the dense preconditioner forms K by a tiled product over R stored densely when that
  // copy stays below 256 MB (else it scans R's rows)
  const bool dense_rd = dense && nR * n <= (int64_t)(32 << 20);   // decided from sizes: a counting
                                                                 // pass returns null pointers
  d.Rd = dense_rd ? cv.take<float2>(nR * n) : nullptr;
  d.wdf = dense ? cv.take<float2>(std::max<int64_t>(nR, 1)) : nullptr;
  {
    const int64_t nt = (n + 31) / 32, splits = gram_splits(n);
    d.gram_part = (dense_rd && splits > 1) ? cv.take<float2>(splits * (nt * (nt + 1) / 2) * 1024) : nullptr;
  }
  d.dense_aux = dense ? cv.take<double>(4) : nullptr;
  d.chol_diag = cv.take<double>(std::max<int64_t>(dense ? n : 0, stiff_cap));
  d.chol_rinv = cv.take<double>(std::max<int64_t>(dense ? n : 0, stiff_cap));
  d.chol_tiles = cv.take<double>(std::max<int64_t>(dense ? (n + 31) / 32 : 0, (stiff_cap + 31) / 32) * 1024);
  d.chol_rdf = dense ? cv.take<float2>(n) : nullptr;
  d.chol_tinv = dense ? cv.take<float2>((n + 31) / 32 * 1024) : nullptr;
  d.storage = storage;
  if (df) {
    d.p_df = cv.take<float2>(n);
    d.v_df = cv.take<float2>(nR);
  } else {
    d.p_df = d.v_df = nullptr;
  }
  if (storage != ST_F64) {
    d.p32 = cv.take<float>((n + 3) & ~int64_t(3));
    d.w32 = cv.take<float>(nR);
    d.dxr = cv.take<double>(n);
  } else {
    d.p32 = d.w32 = nullptr;
    d.dxr = nullptr;
  }
  if (d.ucap) {
    d.U = cv.take<double>(n * d.ucap);
    d.uw = cv.take<double>(d.ucap);
    d.lrs = cv.take<double>(d.ucap);
    d.upart = cv.take<double>((int64_t)d.ublocks * d.ucap);
    d.lrq = cv.take<double>(d.ucap);
  } else {
    d.U = d.uw = d.lrs = d.upart = d.lrq = nullptr;
  }
  if (nblk) {
    d.blkC = cv.take<double>(nblk * 1024);
    d.blkL = cv.take<double>(nblk * 1024);
  } else {
    d.blkC = d.blkL = nullptr;
  }
  d.trace = cv.take<double>((int64_t)trace_cap * kTraceCols);
  d.partials = cv.take<double>(32 * (int64_t)kMaxRedBlocks);
  d.sc = cv.take<Scal>(1);
}

// Stiff-row capacity of a handle and the matching capacity of the stiff CSC lists.
void stiff_caps(const ipm_options& o, int64_t m, const std::vector<int64_t>& sc_prefix, int* stiff_cap,
                int64_t* sc_cap) {
  *stiff_cap = std::max(1, std::min<int>(o.stiff_max > 0 ? o.stiff_max : 1, (int)std::max<int64_t>(m, 1)));
  const int64_t k = std::min<int64_t>(*stiff_cap, (int64_t)sc_prefix.size() - 1);
  *sc_cap = std::max<int64_t>(k > 0 ? sc_prefix[k] : 0, 1);
}

// One device allocation; IPM_ERR_OOM with a message on failure.
int dev_alloc(ipm_handle* h, void** p, size_t bytes, const char* what) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(h, IPM_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes (" + what + ") failed");
  }
  return IPM_OK;
}

// Pinned trace buffer for the rows copied back after each solve.
int alloc_trace(ipm_handle* h) {
  h->trace_cap = h->opt.max_ipm;
  if (cudaMallocHost(&h->htrace, sizeof(double) * kTraceCols * (size_t)h->trace_cap) != cudaSuccess) {
    cudaGetLastError();
    h->htrace = nullptr;
    return fail(h, IPM_ERR_OOM, "pinned trace buffer");
  }
  return IPM_OK;
}

int validate_options(const ipm_options& o) {
  if (!(o.tol_kkt > 0) || !(o.tau > 0 && o.tau < 1) || o.max_ipm < 1 || o.max_cg < 1) return IPM_ERR_ARG;
  if (!(o.cg_eta_min > 0) || !(o.cg_eta_max >= o.cg_eta_min) || !(o.cg_eta_factor > 0)) return IPM_ERR_ARG;
  if (o.precond < 0 || o.precond > 4 || o.stiff_max < 0 || o.stiff_max > 1024) return IPM_ERR_ARG;
  if (o.dense_max_n < 0 || o.dense_max_n > 2048 || !(o.stiff_gamma > 0)) return IPM_ERR_ARG;
  if (o.storage < 0 || o.storage > 3 || o.refine_max < 1 || !(o.refine_eta >= 0 && o.refine_eta < 1)) return IPM_ERR_ARG;
  if (!(o.warm_rho >= 0 && o.warm_rho < 1)) return IPM_ERR_ARG;
  if (o.u_cap < 0 || o.u_cap > (1 << 16)) return IPM_ERR_ARG;
  if (o.system != IPM_SYSTEM_CONDENSED && o.system != IPM_SYSTEM_AUGMENTED) return IPM_ERR_ARG;
  if (o.op_arith < IPM_ARITH_F64 || o.op_arith > IPM_ARITH_MIXED) return IPM_ERR_ARG;
  if (o.rows_format < IPM_ROWS_AUTO || o.rows_format > IPM_ROWS_RUNS) return IPM_ERR_ARG;
  if (o.rows_stage < 0 || o.rows_stage > 1 || !(o.wait_limit_ms > 0 && o.wait_limit_ms <= 6e4)) return IPM_ERR_ARG;
  if (o.wait_test < 0 || o.wait_test > 1 || o.cols_format < 0 || o.cols_format > 1) return IPM_ERR_ARG;
  if (o.refine_mode < 0 || o.refine_mode > 2) return IPM_ERR_ARG;
  if (o.system == IPM_SYSTEM_AUGMENTED &&
      (o.storage != IPM_STORAGE_F64 || (o.precond != IPM_PRECOND_JACOBI && o.precond != IPM_PRECOND_AUTO)))
    return IPM_ERR_ARG;   // the doubly augmented system runs FP64 with the Jacobi preconditioner
  // the dense factor is an FP64 preconditioner for the FP64 operator: with a reduced-precision
  // operator the refinement's inner PCG under it stalled near convergence (RT n = 900, FP8)
  if (o.precond == IPM_PRECOND_DENSE && o.storage != IPM_STORAGE_F64) return IPM_ERR_ARG;
  // likewise the block factors (RT n = 900 with BF16 storage ended in IPM_NUMERICAL)
  if (o.precond == IPM_PRECOND_BLOCK32 && o.storage != IPM_STORAGE_F64) return IPM_ERR_ARG;
  auto lanes_ok = [](int g) { return g == 0 || g == 4 || g == 8 || g == 16 || g == 32; };
  if (!lanes_ok(o.lanes_rows) || !lanes_ok(o.lanes_cols) || !lanes_ok(o.lanes_at)) return IPM_ERR_ARG;
  return IPM_OK;
}

// Host copy of the device scalars (one small D2H plus a synchronisation).
int pull_scal(ipm_handle* h) {
  CUDA_TRY(h, cudaMemcpyAsync(h->hs, h->d.sc, sizeof(Scal), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return IPM_OK;
}

// Orders the internal stream after the caller's stream.
int enter(ipm_handle* h, void* stream) {
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaEventRecord(h->ev, (cudaStream_t)stream));
  CUDA_TRY(h, cudaStreamWaitEvent(h->st, h->ev, 0));
  return IPM_OK;
}

// Orders the caller's stream after the internal stream.
int leave(ipm_handle* h, void* stream) {
  CUDA_TRY(h, cudaEventRecord(h->ev, h->st));
  CUDA_TRY(h, cudaStreamWaitEvent((cudaStream_t)stream, h->ev, 0));
  return IPM_OK;
}

// Lanes per row from the average row length (used when autotuning is off): a group of G
// lanes keeps at most 64 entries per lane (4, 8, 16 or 32 lanes).
int heuristic_group(double avg_nnz) {
  int g = 4;
  while (g < 32 && avg_nnz / g > 64.0) g *= 2;
  return g;
}

// Autotuner results per matrix signature (n, rows of R, non-zeros), process-wide, so that a
// QP loaded again in the same process runs the same schedule (and gives the same bits).
std::mutex g_tune_mu;
std::map<std::tuple<int64_t, int64_t, int64_t>, std::pair<int, int>> g_tune_cache;

// Operator formats decided once R and R^T are on the device: the double-float copies of the
// values (asked for by options.op_arith, kept only when every value is in the float32 range
// the pairs need) and the runs of R's rows (options.rows_format; AUTO takes them when they
// average at least 8 entries).  The runs get a device allocation of their own, sized here.
// The gap layout of R^T for the reduced-precision column pass (options.cols_format = 1): slots
// per column counted on the device, their offsets scanned here, then filled on the device.
int prepare_gap_layout(ipm_handle* h) {
  Dev& d = h->d;
  d.gap = 0;
  d.nslots = 0;
  if (d.storage == ST_F64 || h->opt.cols_format != 1 || d.nnzR == 0) return IPM_OK;
  int32_t* cnt = reinterpret_cast<int32_t*>(d.tR);     // nR doubles of iteration work space
  std::vector<int32_t> hc((size_t)d.n);
  if (d.nR * 2 >= d.n) {
    CUDA_TRY(h, launch_gap_count(d, cnt, h->st));
  } else {
    return IPM_OK;                                     // no room for the counts (fewer rows than n / 2)
  }
  CUDA_TRY(h, cudaMemcpyAsync(hc.data(), cnt, sizeof(int32_t) * hc.size(), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  std::vector<int64_t> gp((size_t)d.n + 1, 0);
  for (int64_t j = 0; j < d.n; ++j) gp[j + 1] = gp[j] + hc[j];
  const int64_t ns = gp[d.n];
  const int vb = d.storage == ST_F32 ? 4 : d.storage == ST_BF16 ? 2 : 1;
  Carver cc(nullptr);
  cc.take<int64_t>(d.n + 1);
  cc.take<int32_t>(d.n);
  cc.take<uint16_t>(ns);
  cc.take<unsigned char>((int64_t)vb * ns);
  const size_t bytes = cc.off + 256;
  if (h->opt.mem_budget > 0 && (double)(h->mat->bytes + h->arena_bytes + bytes) > h->opt.mem_budget)
    return IPM_OK;                                     // within the budget the column pass stays CSR
  int rc;
  if ((rc = dev_alloc(h, &h->mat->gap, bytes, "gap layout of R^T"))) return rc;
  h->mat->bytes += bytes;
  Carver cv((char*)h->mat->gap);
  d.gp_ptr = cv.take<int64_t>(d.n + 1);
  d.gp_base = cv.take<int32_t>(d.n);
  d.gp_d = cv.take<uint16_t>(ns);
  d.gp_q = cv.take<unsigned char>((int64_t)vb * ns);
  d.nslots = ns;
  CUDA_TRY(h, cudaMemcpyAsync((void*)d.gp_ptr, gp.data(), sizeof(int64_t) * gp.size(), cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, launch_gap_fill(d, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  d.gap = 1;
  return IPM_OK;
}

int prepare_operator_formats(ipm_handle* h) {
  Dev& d = h->d;
  d.df = 0;
  d.mx = 0;
  {
    const int rc0 = prepare_gap_layout(h);
    if (rc0) return rc0;
  }
  if (d.R_df) {
    int* flag = reinterpret_cast<int*>(d.partials);   // reduction scratch, free at set-up
    CUDA_TRY(h, cudaMemsetAsync(flag, 0, sizeof(int), h->st));
    CUDA_TRY(h, launch_df_split(d, flag, h->st));
    int bad = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    d.df = (!bad && h->opt.op_arith == IPM_ARITH_DF32) ? 1 : 0;
    d.mx = (!bad && h->opt.op_arith == IPM_ARITH_MIXED) ? 1 : 0;
  }
  d.runs = 0;
  d.ntiles = 0;
  d.tile_row = nullptr;
  d.wait_ns = (uint64_t)(h->opt.wait_limit_ms * 1e6);
  d.wait_test = h->opt.wait_test;
  d.npieces = 0;
  d.pc_ptr = nullptr;
  d.pc_col = nullptr;
  d.pc_ol = nullptr;
  // (the split-pipe passes read R's rows as CSR)
  if (h->opt.rows_format == IPM_ROWS_CSR || d.mx || d.nR == 0 || d.nnzR == 0) return IPM_OK;
  // per row: runs and pieces (two int32 per row in the nR doubles of iteration work space tR)
  int32_t* cnt = reinterpret_cast<int32_t*>(d.tR);
  CUDA_TRY(h, launch_runs_count(d, cnt, cnt + d.nR, h->st));
  std::vector<int32_t> hc(2 * (size_t)d.nR);
  std::vector<int64_t> rows(d.nR + 1);
  CUDA_TRY(h, cudaMemcpyAsync(hc.data(), cnt, sizeof(int32_t) * hc.size(), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(rows.data(), d.R_ptr, sizeof(int64_t) * rows.size(), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  std::vector<int64_t> pp((size_t)d.nR + 1, 0);
  int64_t nruns = 0, longest = 0;
  for (int64_t r = 0; r < d.nR; ++r) {
    nruns += hc[r];
    pp[r + 1] = pp[r] + hc[d.nR + r];
    longest = std::max<int64_t>(longest, rows[r + 1] - rows[r]);
  }
  const int64_t npieces = pp[d.nR];
  // a piece records its offset in the row in 26 bits
  if (nruns == 0 || longest >= ((int64_t)1 << 26)) return IPM_OK;
  const bool use = h->opt.rows_format == IPM_ROWS_RUNS ||
                   (d.storage != ST_F64 && (double)d.nnzR >= 8.0 * (double)nruns);
  if (!use) return IPM_OK;
  // tiles of the staged rows pass (double-float or reduced storage): consecutive rows, at most
  // one per lane group (32 rows for double-float, 64 otherwise), whose values take at most
  // kStageValBytes - 16 bytes and whose pieces number at most kStagePieces (so the
  // 16-byte-aligned spans fit a stage); a row beyond that is a tile of its own, read from
  // global memory
  std::vector<int32_t> tiles;
  const int vbytes = d.df ? 8 : (d.storage == ST_F32 ? 4 : d.storage == ST_BF16 ? 2 : d.storage == ST_FP8 ? 1 : 0);
  if (vbytes && h->opt.rows_stage == 1) {
    const int64_t cap = (kStageValBytes - 16) / vbytes;
    const int64_t max_rows = d.df ? kStagedThreads / 16 : kStagedThreads / 8;
    tiles.push_back(0);
    int64_t r = 0;
    while (r < d.nR) {
      int64_t r1 = r + 1;
      while (r1 < d.nR && r1 - r < max_rows && rows[r1 + 1] - rows[r] <= cap && pp[r1 + 1] - pp[r] <= kStagePieces) ++r1;
      tiles.push_back((int32_t)r1);
      r = r1;
    }
  }
  const int64_t ntiles = tiles.empty() ? 0 : (int64_t)tiles.size() - 1;
  Carver cc(nullptr);
  cc.take<int64_t>(d.nR + 1);
  cc.take<int32_t>(npieces);
  cc.take<uint32_t>(npieces);
  cc.take<int32_t>(ntiles + 1);
  const size_t bytes = cc.off + 256;
  if (h->opt.mem_budget > 0 && (double)(h->mat->bytes + h->arena_bytes + bytes) > h->opt.mem_budget)
    return IPM_OK;                                     // within the budget the rows pass stays CSR
  int rc;
  if ((rc = dev_alloc(h, &h->mat->aux, bytes, "pieces of R's runs"))) return rc;
  h->mat->bytes += bytes;
  Carver cv((char*)h->mat->aux);
  d.pc_ptr = cv.take<int64_t>(d.nR + 1);
  d.pc_col = cv.take<int32_t>(npieces);
  d.pc_ol = cv.take<uint32_t>(npieces);
  d.tile_row = cv.take<int32_t>(ntiles + 1);
  d.npieces = npieces;
  if (ntiles) {
    CUDA_TRY(h, prepare_staged());
    CUDA_TRY(h, cudaMemcpyAsync((void*)d.tile_row, tiles.data(), sizeof(int32_t) * tiles.size(), cudaMemcpyHostToDevice, h->st));
  }
  CUDA_TRY(h, cudaMemcpyAsync((void*)d.pc_ptr, pp.data(), sizeof(int64_t) * pp.size(), cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, launch_runs_fill(d, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  d.ntiles = ntiles;
  d.runs = 1;
  return IPM_OK;
}

// Segments of the block-Jacobi preconditioner: for every row of R, the maximal stretches of its
// entries whose columns fall into one block of 32 variables (the columns of a row must
// increase), listed block by block in row order (a stable counting sort by block), once for
// every row and once for the constraint rows; then the part of the blocks fixed for the QP.
int prepare_block_segments(ipm_handle* h, const std::vector<int64_t>& Rp, const std::vector<int32_t>& arow) {
  Dev& d = h->d;
  d.nblk = (d.n + 31) / 32;
  std::vector<int32_t> ri((size_t)d.nnzR);
  if (d.nnzR) {
    CUDA_TRY(h, cudaMemcpyAsync(ri.data(), d.R_idx, sizeof(int32_t) * ri.size(), cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
  }
  std::vector<unsigned char> is_con((size_t)std::max<int64_t>(d.nR, 1), 0);
  for (int32_t r : arow) is_con[r] = 1;
  // count segments per block (all rows, constraint rows)
  std::vector<int64_t> cs(d.nblk + 1, 0), cc(d.nblk + 1, 0);
  for (int64_t r = 0; r < d.nR; ++r)
    for (int64_t e = Rp[r]; e < Rp[r + 1]; ++e) {
      if (e > Rp[r] && ri[e] <= ri[e - 1])
        return fail(h, IPM_ERR_ARG, "BLOCK32 needs the columns of every row in increasing order");
      if (e == Rp[r] || ri[e] / 32 != ri[e - 1] / 32) {
        cs[ri[e] / 32 + 1]++;
        if (is_con[r]) cc[ri[e] / 32 + 1]++;
      }
    }
  for (int64_t b = 0; b < d.nblk; ++b) {
    cs[b + 1] += cs[b];
    cc[b + 1] += cc[b];
  }
  const int64_t ns = cs[d.nblk], nc = cc[d.nblk];
  std::vector<int32_t> srow(ns), scnt(ns), crow(nc), ccnt(nc);
  std::vector<int64_t> sbeg(ns), cbeg(nc);
  std::vector<int64_t> fs(cs.begin(), cs.end() - 1), fc(cc.begin(), cc.end() - 1);
  for (int64_t r = 0; r < d.nR; ++r) {
    int64_t e = Rp[r];
    while (e < Rp[r + 1]) {
      const int32_t b = ri[e] / 32;
      int64_t f = e + 1;
      while (f < Rp[r + 1] && ri[f] / 32 == b) ++f;
      const int64_t k = fs[b]++;
      srow[k] = (int32_t)r; sbeg[k] = e; scnt[k] = (int32_t)(f - e);
      if (is_con[r]) {
        const int64_t kc = fc[b]++;
        crow[kc] = (int32_t)r; cbeg[kc] = e; ccnt[kc] = (int32_t)(f - e);
      }
      e = f;
    }
  }
  Carver cc0(nullptr);
  cc0.take<int64_t>(d.nblk + 1); cc0.take<int64_t>(ns); cc0.take<int32_t>(ns); cc0.take<int32_t>(ns);
  cc0.take<int64_t>(d.nblk + 1); cc0.take<int64_t>(nc); cc0.take<int32_t>(nc); cc0.take<int32_t>(nc);
  const size_t bytes = cc0.off + 256;
  int rc;
  if ((rc = dev_alloc(h, &h->mat->blk, bytes, "block-Jacobi segments"))) return rc;
  h->mat->bytes += bytes;
  Carver cv((char*)h->mat->blk);
  d.bs_ptr = cv.take<int64_t>(d.nblk + 1); d.bs_beg = cv.take<int64_t>(ns);
  d.bs_row = cv.take<int32_t>(ns); d.bs_cnt = cv.take<int32_t>(ns);
  d.bc_ptr = cv.take<int64_t>(d.nblk + 1); d.bc_beg = cv.take<int64_t>(nc);
  d.bc_row = cv.take<int32_t>(nc); d.bc_cnt = cv.take<int32_t>(nc);
  auto up = [&](const void* dst, const void* src, size_t nb) -> int {
    if (nb) CUDA_TRY(h, cudaMemcpyAsync((void*)dst, src, nb, cudaMemcpyHostToDevice, h->st));
    return IPM_OK;
  };
  if ((rc = up(d.bs_ptr, cs.data(), 8 * cs.size())) || (rc = up(d.bs_beg, sbeg.data(), 8 * sbeg.size())) ||
      (rc = up(d.bs_row, srow.data(), 4 * srow.size())) || (rc = up(d.bs_cnt, scnt.data(), 4 * scnt.size())) ||
      (rc = up(d.bc_ptr, cc.data(), 8 * cc.size())) || (rc = up(d.bc_beg, cbeg.data(), 8 * cbeg.size())) ||
      (rc = up(d.bc_row, crow.data(), 4 * crow.size())) || (rc = up(d.bc_cnt, ccnt.data(), 4 * ccnt.size())))
    return rc;
  CUDA_TRY(h, launch_block_const(d, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));   // host staging buffers go out of scope
  return IPM_OK;
}

// Times the two operator kernels for every lane-group size on the loaded matrices (three
// launches each after one warm-up, CUDA events on the handle's stream) and keeps the fastest.
int autotune_groups(ipm_handle* h) {
  Dev& d = h->d;
  const auto key = std::make_tuple(d.n, d.nR, d.nnzR);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      d.g_rows = it->second.first;
      d.g_cols = it->second.second;
      h->g = make_geo(d);
      return IPM_OK;
    }
  }
  CUDA_TRY(h, cudaMemsetAsync(d.p, 0, sizeof(double) * d.n, h->st));
  if (d.p_df) CUDA_TRY(h, cudaMemsetAsync(d.p_df, 0, sizeof(float2) * d.n, h->st));
  if (d.v_df && d.nR) CUDA_TRY(h, cudaMemsetAsync(d.v_df, 0, sizeof(float2) * d.nR, h->st));
  CUDA_TRY(h, cudaMemsetAsync(d.sigma, 0, sizeof(double) * d.n, h->st));
  if (d.nR) {
    CUDA_TRY(h, cudaMemsetAsync(d.omega, 0, sizeof(double) * d.nR, h->st));
    CUDA_TRY(h, cudaMemsetAsync(d.vR, 0, sizeof(double) * d.nR, h->st));
  }
  cudaEvent_t e0, e1;
  CUDA_TRY(h, cudaEventCreate(&e0));
  CUDA_TRY(h, cudaEventCreate(&e1));
  const int cand[4] = {4, 8, 16, 32};
  for (int which = 0; which < 2; ++which) {
    if (which == 0 && d.nR == 0) continue;
    float best = 1e30f;
    int bestg = which == 0 ? d.g_rows : d.g_cols;
    for (int gsz : cand) {
      if (which == 0) d.g_rows = gsz; else d.g_cols = gsz;
      const Geo g = make_geo(d);
      auto run = [&]() { return which == 0 ? launch_op_rows_only(d, g, h->st) : launch_op_cols_only(d, g, h->st); };
      CUDA_TRY(h, run());
      CUDA_TRY(h, cudaEventRecord(e0, h->st));
      for (int r = 0; r < 3; ++r) CUDA_TRY(h, run());
      CUDA_TRY(h, cudaEventRecord(e1, h->st));
      CUDA_TRY(h, cudaEventSynchronize(e1));
      float ms = 0;
      CUDA_TRY(h, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; bestg = gsz; }
    }
    if (which == 0) d.g_rows = bestg; else d.g_cols = bestg;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->g = make_geo(d);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = std::make_pair(d.g_rows, d.g_cols);
  return IPM_OK;
}

// Adds a conditional while node at the current capture point of `st` (default condition 1,
// reset at every graph launch) and captures its body on `body_st` with fill(handle, body_st).
// A handle created here is reset to 1 at every launch of the top-level graph only; a loop
// nested in another loop's body must have its condition set by a kernel before each entry
// (pass that handle in `pre`, created with new_handle()).
cudaError_t new_handle(cudaStream_t st, cudaGraphConditionalHandle* ch) {
  cudaStreamCaptureStatus cs;
  unsigned long long cid;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, &cid, &cg, &deps, &edata, &ndeps);
  if (e != cudaSuccess) return e;
  return cudaGraphConditionalHandleCreate(ch, cg, 1u, cudaGraphCondAssignDefault);
}

template <typename Fill>
cudaError_t add_while(cudaStream_t st, cudaStream_t body_st, Fill fill, int* body_kernels,
                      const cudaGraphConditionalHandle* pre = nullptr) {
  cudaStreamCaptureStatus cs;
  unsigned long long cid;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, &cid, &cg, &deps, &edata, &ndeps);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
  cudaGraphConditionalHandle ch = 0;
  if (pre) {
    ch = *pre;
  } else {
    e = cudaGraphConditionalHandleCreate(&ch, cg, 1u, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
  }
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = ch;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode = nullptr;
  e = cudaGraphAddNode(&cnode, cg, dv.data(), nullptr, dv.size(), &cp);
  if (e != cudaSuccess) return e;
  e = cudaStreamUpdateCaptureDependencies(st, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(body_st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t ef = fill(ch, body_st);
  cudaGraph_t bodyo = nullptr;
  e = cudaStreamEndCapture(body_st, &bodyo);
  if (ef != cudaSuccess) return ef;
  if (e != cudaSuccess) return e;
  if (body_kernels) *body_kernels = count_kernel_nodes(body);
  return cudaSuccess;
}

// Reduced storage: whether a Newton step runs one PCG with residual replacement (refine_mode 1,
// or 2 = automatic: replacement for F32 and BF16; FP8's coarse values let the kept direction
// drift, so it takes restarted passes) and the factor between FP64 residual evaluations
// (refine_eta, 0 = automatic: 0.01 with replacement, 0.1 with passes).
bool refine_replaces(const ipm_handle* h) {
  const int m = h->opt.refine_mode;
  return m == 1 || (m == 2 && h->opt.storage != IPM_STORAGE_FP8_E4M3);
}

double refine_factor(const ipm_handle* h) {
  if (h->opt.refine_eta > 0) return h->opt.refine_eta;
  return refine_replaces(h) ? 0.01 : 0.1;
}

// Emits (into the capture running on `st`) one Newton step -- diagonal update, preconditioner,
// right-hand side, PCG (nested while loops; with a reduced-precision store the PCG loop sits in
// an FP64 refinement loop followed by an FP64 fallback loop) and direction recovery -- and,
// when `full`, the ratio test, update, residual summary and control.  Nested loops are re-armed
// by a kernel before each entry (their default is applied only at top-level graph launch).
// Side streams s2, s3 capture the loop bodies.  `ipm_loop` is the handle the control kernel
// sets (0: none).
cudaError_t emit_step(ipm_handle* h, int pc, bool full, cudaStream_t st, cudaStream_t s2, cudaStream_t s3,
                      cudaGraphConditionalHandle ipm_loop, LoopCounts* c) {
  const Dev& d = h->d;
  const Geo& g = h->g;
  const bool lowp = d.storage != ST_F64;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess && x != cudaSuccess) e = x; };
  chk(launch_diag_update(d, g, st));
  chk(launch_precond_build(d, g, pc, st));
  chk(launch_rhs(d, g, pc, st));
  chk(launch_precond_finish(d, g, pc, st));
  if (!lowp) {
    cudaGraphConditionalHandle hp = 0;
    chk(new_handle(st, &hp));
    chk(launch_set_cond(hp, 1u, st));
    chk(launch_cg_init(d, g, pc, st));
    if (e == cudaSuccess)
      chk(add_while(st, s2, [&](cudaGraphConditionalHandle ch, cudaStream_t bs) {
            return launch_cg_body(d, g, pc, ch, bs, true, false);
          }, &c->pcg, &hp));
  } else if (refine_replaces(h)) {
    // one reduced-precision PCG with residual replacement, then the FP64 fallback
    cudaGraphConditionalHandle hp = 0, hf = 0;
    chk(new_handle(st, &hp));
    chk(new_handle(st, &hf));
    chk(launch_ru_start(d, st));
    chk(launch_set_cond(hp, 1u, st));
    chk(launch_cg_init(d, g, pc, st));
    c->ru = 1;
    if (e == cudaSuccess)
      chk(add_while(st, s2, [&](cudaGraphConditionalHandle ch, cudaStream_t bs) {
            return launch_ru_body(d, g, pc, ch, bs, true);
          }, &c->pcg, &hp));
    chk(launch_ru_end(d, g, st));
    chk(launch_refine_fallback(d, g, st));
    chk(launch_set_cond(hf, 1u, st));
    chk(launch_cg_init(d, g, pc, st));
    if (e == cudaSuccess)
      chk(add_while(st, s2, [&](cudaGraphConditionalHandle ch, cudaStream_t bs) {
            return launch_cg_body(d, g, pc, ch, bs, true, false);
          }, &c->fallback, &hf));
    chk(launch_refine_finish(d, g, st));
  } else {
    cudaGraphConditionalHandle hr = 0, hf = 0;
    chk(new_handle(st, &hr));
    chk(new_handle(st, &hf));
    chk(launch_refine_start(d, g, st));
    chk(launch_set_cond(hr, 1u, st));
    if (e == cudaSuccess)
      chk(add_while(st, s2, [&](cudaGraphConditionalHandle ho, cudaStream_t bs) {
            cudaGraphConditionalHandle hi = 0;
            cudaError_t x = new_handle(bs, &hi);
            if (x == cudaSuccess) x = launch_refine_inner(d, g, hi, bs);
            if (x == cudaSuccess) x = launch_cg_init(d, g, pc, bs);
            if (x == cudaSuccess)
              x = add_while(bs, s3, [&](cudaGraphConditionalHandle hin, cudaStream_t bs2) {
                    return launch_cg_body(d, g, pc, hin, bs2, true, true);
                  }, &c->pcg, &hi);
            if (x == cudaSuccess) x = launch_refine_tail(d, g, ho, bs);
            return x;
          }, &c->refine, &hr));
    // FP64 fallback for a step the refinement could not finish (exits at once otherwise)
    chk(launch_refine_fallback(d, g, st));
    chk(launch_set_cond(hf, 1u, st));
    chk(launch_cg_init(d, g, pc, st));
    if (e == cudaSuccess)
      chk(add_while(st, s2, [&](cudaGraphConditionalHandle ch, cudaStream_t bs) {
            return launch_cg_body(d, g, pc, ch, bs, true, false);
          }, &c->fallback, &hf));
    chk(launch_refine_finish(d, g, st));
  }
  chk(launch_recover(d, g, st));
  if (full) {
    chk(launch_ratio(d, g, st));
    chk(launch_update(d, g, st));
    chk(launch_residual_summary(d, g, st));
    chk(launch_control(d, st, ipm_loop));
  }
  return e;
}

// Emits a whole solve into the capture on `st`: start point (cold) or residual summary +
// warm mu (warm), totals reset, then the IPM while loop around emit_step.
cudaError_t emit_solve(ipm_handle* h, int pc, bool warm, cudaStream_t st, LoopCounts* c) {
  const Dev& d = h->d;
  const Geo& g = h->g;
  cudaError_t e = warm ? launch_warm_start(d, g, st) : launch_start_point(d, g, st);
  if (e == cudaSuccess) e = launch_solve_begin(d, st);
  if (e == cudaSuccess)
    e = add_while(st, h->st2, [&](cudaGraphConditionalHandle hipm, cudaStream_t bs) {
          return emit_step(h, pc, true, bs, h->st3, h->st4, hipm, c);
        }, &c->ipm);
  return e;
}

int finish_capture(ipm_handle* h, cudaError_t e, cudaStream_t st, cudaGraphExec_t* out, cudaGraph_t* keep, int* top) {
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(st, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess && top) *top = count_kernel_nodes(graph);
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
  if (graph) {
    if (keep && e == cudaSuccess) *keep = graph;
    else cudaGraphDestroy(graph);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, IPM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  return IPM_OK;
}

int ensure_solve_graph(ipm_handle* h, int pc, bool warm) {
  Graphs& gr = h->graphs[pc];
  const int w = warm ? 1 : 0;
  if (gr.solve[w]) return IPM_OK;
  gr.solve_c[w] = LoopCounts{};
  CUDA_TRY(h, cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = emit_solve(h, pc, warm, h->st, &gr.solve_c[w]);
  return finish_capture(h, e, h->st, &gr.solve[w], &gr.solve_g[w], &gr.solve_c[w].top);
}

int ensure_dir_graph(ipm_handle* h, int pc) {
  Graphs& gr = h->graphs[pc];
  if (gr.dir) return IPM_OK;
  gr.dir_c = LoopCounts{};
  CUDA_TRY(h, cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = emit_step(h, pc, false, h->st, h->st2, h->st3, 0, &gr.dir_c);
  return finish_capture(h, e, h->st, &gr.dir, nullptr, &gr.dir_c.top);
}

// One IPM iteration with every kernel launched directly (use_graphs = 0): the same sequence
// as the captured graph, with the loops driven from the host (one scalar read per trip).
// Adds the kernels it launched to *launches.
int run_iteration_direct(ipm_handle* h, int pc, int64_t* launches) {
  const Dev& d = h->d;
  const Geo& g = h->g;
  cudaStream_t st = h->st;
  const LoopCounts& lc = h->graphs[pc].solve_c[0];
  auto pcg = [&](bool lowp) -> int {
    int done = 0;
    for (int k = 0; k < h->opt.max_cg + 1 && !done; ++k) {
      CUDA_TRY(h, launch_cg_body(d, g, pc, 0, st, false, lowp));
      CUDA_TRY(h, cudaMemcpyAsync(&h->hs->cg_done, &d.sc->cg_done, sizeof(int), cudaMemcpyDeviceToHost, st));
      CUDA_TRY(h, cudaStreamSynchronize(st));
      done = h->hs->cg_done;
      *launches += lowp ? lc.pcg : lc.pcg;
    }
    return IPM_OK;
  };
  CUDA_TRY(h, launch_diag_update(d, g, st));
  CUDA_TRY(h, launch_precond_build(d, g, pc, st));
  CUDA_TRY(h, launch_rhs(d, g, pc, st));
  CUDA_TRY(h, launch_precond_finish(d, g, pc, st));
  int rc;
  if (d.storage == ST_F64) {
    CUDA_TRY(h, launch_cg_init(d, g, pc, st));
    if ((rc = pcg(false))) return rc;
  } else if (refine_replaces(h)) {
    CUDA_TRY(h, launch_ru_start(d, st));
    CUDA_TRY(h, launch_cg_init(d, g, pc, st));
    int done = 0;
    for (int k = 0; k < h->opt.max_cg + 1 && !done; ++k) {
      CUDA_TRY(h, launch_ru_body(d, g, pc, 0, st, false));
      CUDA_TRY(h, cudaMemcpyAsync(&h->hs->cg_done, &d.sc->cg_done, sizeof(int), cudaMemcpyDeviceToHost, st));
      CUDA_TRY(h, cudaStreamSynchronize(st));
      done = h->hs->cg_done;
      *launches += lc.pcg;
    }
    CUDA_TRY(h, launch_ru_end(d, g, st));
    CUDA_TRY(h, launch_refine_fallback(d, g, st));
    CUDA_TRY(h, launch_cg_init(d, g, pc, st));
    if ((rc = pcg(false))) return rc;
    CUDA_TRY(h, launch_refine_finish(d, g, st));
  } else {
    CUDA_TRY(h, launch_refine_start(d, g, st));
    for (int it = 0; it < h->opt.refine_max; ++it) {
      CUDA_TRY(h, launch_refine_inner(d, g, 0, st));
      CUDA_TRY(h, launch_cg_init(d, g, pc, st));
      if ((rc = pcg(true))) return rc;
      CUDA_TRY(h, launch_refine_tail(d, g, 0, st));
      *launches += lc.refine;
      CUDA_TRY(h, cudaMemcpyAsync(h->hs, d.sc, sizeof(Scal), cudaMemcpyDeviceToHost, st));
      CUDA_TRY(h, cudaStreamSynchronize(st));
      if (h->hs->cg_conv_outer || !std::isfinite(h->hs->rr_outer)) break;
    }
    CUDA_TRY(h, launch_refine_fallback(d, g, st));
    CUDA_TRY(h, launch_cg_init(d, g, pc, st));
    if ((rc = pcg(false))) return rc;
    CUDA_TRY(h, launch_refine_finish(d, g, st));
  }
  CUDA_TRY(h, launch_recover(d, g, st));
  CUDA_TRY(h, launch_ratio(d, g, st));
  CUDA_TRY(h, launch_update(d, g, st));
  CUDA_TRY(h, launch_residual_summary(d, g, st));
  CUDA_TRY(h, launch_control(d, st));
  *launches += lc.ipm;
  return IPM_OK;
}

int choose_precond(const ipm_handle* h) {
  const ipm_options& o = h->opt;
  int pc = o.precond;
  if (o.system == IPM_SYSTEM_AUGMENTED) return PC_JACOBI;   // the paper's Jacobi PCG on eq:2x2_augmented
  if (pc == IPM_PRECOND_BLOCK32) return h->d.nblk ? PC_BLOCK32 : PC_JACOBI_LR;   // segments come from ipm_set_qp
  if (pc == IPM_PRECOND_AUTO) pc = (h->d.Kd && h->d.n <= 1024) ? PC_DENSE : PC_JACOBI_LR;
  if (pc == PC_DENSE && !h->d.Kd) pc = PC_JACOBI_LR;
  return pc;
}

// Writes the solver options into the device scalars (keeps the iterate state).
int push_options(ipm_handle* h) {
  Scal& s = *h->hs;
  s.tol_kkt = h->opt.tol_kkt;
  s.tau = h->opt.tau;
  s.max_ipm = h->opt.max_ipm;
  s.cg_max = h->opt.max_cg;
  s.eta_factor = h->opt.cg_eta_factor;
  s.eta_min = h->opt.cg_eta_min;
  s.eta_max = h->opt.cg_eta_max;
  s.stiff_gamma = h->opt.stiff_gamma;
  s.stiff_max = std::min(h->opt.stiff_max, h->d.stiff_cap);
  s.equal_steps = h->opt.equal_steps;
  s.refine_max = h->opt.refine_max;
  s.refine_eta = refine_factor(h);
  s.warm_rho = h->opt.warm_rho;
  s.cnorm = h->cnorm;
  s.bnorm = h->bnorm;
  s.ncomp = h->ncomp;
  return IPM_OK;
}

int copy_out(ipm_handle* h, double* dst, const double* src, int64_t n, int mem) {
  if (!dst || n <= 0) return IPM_OK;
  CUDA_TRY(h, cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)n,
                              mem == IPM_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
  return IPM_OK;
}

int copy_in(ipm_handle* h, double* dst, const double* src, int64_t n, int mem) {
  if (n <= 0) return IPM_OK;
  if (!src) return fail(h, IPM_ERR_ARG, "missing vector");
  CUDA_TRY(h, cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)n,
                              mem == IPM_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
  return IPM_OK;
}

// Scalar fields of the device struct (written from the host between graph launches).
int set_scal_double(ipm_handle* h, double* field_dev, double v) {
  CUDA_TRY(h, cudaMemcpyAsync(field_dev, &v, sizeof(double), cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return IPM_OK;
}

}  // namespace

extern "C" {

void ipm_default_options(ipm_options* o) {
  if (!o) return;
  o->tol_kkt = 1e-6;
  o->tau = 0.995;
  o->max_ipm = 200;
  o->max_cg = 2000;
  o->cg_eta_max = 1e-2;
  o->cg_eta_min = 1e-10;
  o->cg_eta_factor = 0.3;
  o->precond = IPM_PRECOND_AUTO;
  o->stiff_gamma = 1.0;
  o->stiff_max = 256;
  o->dense_max_n = 2048;
  o->timeout_ms = 0.0;
  o->mem_budget = 0.0;
  o->equal_steps = 0;
  o->autotune = 0;
  o->use_graphs = 1;
  o->storage = IPM_STORAGE_F64;
  o->refine_max = 8;
  o->refine_eta = 0.0;
  o->lanes_rows = 0;
  o->lanes_cols = 0;
  o->lanes_at = 0;
  o->op_arith = IPM_ARITH_F64;
  o->rows_format = IPM_ROWS_AUTO;
  o->rows_stage = 0;
  o->cols_format = 0;
  o->refine_mode = 2;
  o->wait_limit_ms = 1000.0;
  o->wait_test = 0;
  o->warm_rho = 1e-5;
  o->u_cap = 0;
  o->ingest_host = 0;
  o->system = IPM_SYSTEM_CONDENSED;
}

const char* ipm_status_str(int s) {
  switch (s) {
    case IPM_OK: return "ok";
    case IPM_ERR_ARG: return "invalid argument";
    case IPM_ERR_OOM: return "out of device memory (or over budget)";
    case IPM_MAX_ITER: return "IPM iteration limit reached";
    case IPM_CG_STALL: return "PCG iteration limit reached";
    case IPM_NUMERICAL: return "numerical failure (NaN/Inf or breakdown)";
    case IPM_INFEASIBLE_SUSPECTED: return "problem looks infeasible";
    case IPM_ERR_TIMEOUT: return "wall-clock limit exceeded";
    case IPM_ERR_CUDA: return "CUDA error";
    case IPM_ERR_STATE: return "call out of order";
    case IPM_ERR_TOO_LARGE: return "size exceeds the fixed static scratch (IPM_STATIC_SCRATCH_ROWS rows)";
    default: return "unknown status";
  }
}

const char* ipm_last_error(const ipm_handle* h) { return h ? h->err.c_str() : "null handle"; }

int ipm_create(const ipm_options* opt, ipm_handle** out) {
  if (!out) return IPM_ERR_ARG;
  *out = nullptr;
  ipm_options o;
  ipm_default_options(&o);
  if (opt) o = *opt;
  if (validate_options(o) != IPM_OK) return IPM_ERR_ARG;
  ipm_handle* h = new (std::nothrow) ipm_handle();
  if (!h) return IPM_ERR_OOM;
  h->opt = o;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->st2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->st3, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->st4, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&h->hs, sizeof(Scal)) != cudaSuccess) {
    cudaGetLastError();
    if (h->st) cudaStreamDestroy(h->st);
    if (h->st2) cudaStreamDestroy(h->st2);
    if (h->st3) cudaStreamDestroy(h->st3);
    if (h->st4) cudaStreamDestroy(h->st4);
    if (h->ev) cudaEventDestroy(h->ev);
    delete h;
    return IPM_ERR_CUDA;
  }
  std::memset(h->hs, 0, sizeof(Scal));
  *out = h;
  return IPM_OK;
}

int ipm_update_costs(ipm_handle* h, const double* f_w, const double* c, int mem, void* stream) {
  if (!h) return IPM_ERR_ARG;
  if (!h->loaded) return fail(h, IPM_ERR_STATE, "ipm_update_costs before ipm_set_qp");
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is in flight on this handle");
  int rc;
  const Dev& d = h->d;
  const int64_t fr = h->fr;
  std::vector<double> hw, hc;
  if (f_w && (rc = fetch(h, f_w, fr, mem, hw))) return rc;
  if (c && (rc = fetch(h, c, d.n, mem, hc))) return rc;
  for (double v : hw) if (!std::isfinite(v) || v < 0) return fail(h, IPM_ERR_ARG, "f_w must be finite and >= 0");
  double cn = h->cnorm;
  if (c) {
    cn = 0;
    for (double v : hc) { if (!std::isfinite(v)) return fail(h, IPM_ERR_ARG, "c not finite"); cn = std::max(cn, std::fabs(v)); }
  }
  if ((rc = enter(h, stream))) return rc;
  if (f_w && fr) CUDA_TRY(h, cudaMemcpyAsync((void*)d.wR, hw.data(), 8 * fr, cudaMemcpyHostToDevice, h->st));
  if (c) CUDA_TRY(h, cudaMemcpyAsync((void*)d.c, hc.data(), 8 * d.n, cudaMemcpyHostToDevice, h->st));
  if (f_w) CUDA_TRY(h, launch_diagH(d, h->st));
  if (f_w && d.nblk) CUDA_TRY(h, launch_block_const(d, h->st));   // the blocks' fixed part has w in it
  CUDA_TRY(h, cudaStreamSynchronize(h->st));   // host staging buffers go out of scope
  h->cnorm = cn;
  return leave(h, stream);
}

int ipm_set_lowrank(ipm_handle* h, int64_t u_cols, const double* U, const double* u_w, int mem, void* stream) {
  if (!h) return IPM_ERR_ARG;
  if (!h->loaded) return fail(h, IPM_ERR_STATE, "ipm_set_lowrank before ipm_set_qp");
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is in flight on this handle");
  Dev& d = h->d;
  if (u_cols < 0) return fail(h, IPM_ERR_ARG, "u_cols < 0");
  if (u_cols > d.ucap)
    return fail(h, IPM_ERR_TOO_LARGE, "u_cols " + std::to_string(u_cols) + " above the capacity " +
                                          std::to_string(d.ucap) + " reserved at ipm_set_qp (options.u_cap)");
  if (u_cols && (!U || !u_w)) return fail(h, IPM_ERR_ARG, "u_cols > 0 needs U and u_w");
  int rc;
  std::vector<double> hu, hw;
  if (u_cols) {
    hu.resize((size_t)(d.n * u_cols));
    if ((rc = fetch_into(h, U, d.n * u_cols, mem, hu.data()))) return rc;
    if ((rc = fetch(h, u_w, u_cols, mem, hw))) return rc;
    for (double v : hw) if (!std::isfinite(v)) return fail(h, IPM_ERR_ARG, "u_w not finite");
    for (double v : hu) if (!std::isfinite(v)) return fail(h, IPM_ERR_ARG, "U not finite");
  }
  if ((rc = enter(h, stream))) return rc;
  if (u_cols) {
    CUDA_TRY(h, cudaMemcpyAsync(d.U, hu.data(), 8 * hu.size(), cudaMemcpyHostToDevice, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(d.uw, hw.data(), 8 * hw.size(), cudaMemcpyHostToDevice, h->st));
  }
  d.ucols = u_cols;
  destroy_graphs(h);                    // the captured kernels carry the old column count
  CUDA_TRY(h, launch_diagH(d, h->st));
  if (d.nblk) CUDA_TRY(h, launch_block_const(d, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));   // host staging buffers go out of scope
  return leave(h, stream);
}

int ipm_autotune_reset(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.clear();
  return IPM_OK;
}

int ipm_abi_sizes(int64_t* options, int64_t* qp, int64_t* info, int64_t* cg_report) {
  if (options) *options = (int64_t)sizeof(ipm_options);
  if (qp) *qp = (int64_t)sizeof(ipm_qp);
  if (info) *info = (int64_t)sizeof(ipm_info);
  if (cg_report) *cg_report = (int64_t)sizeof(ipm_cg_report);
  return IPM_OK;
}

int ipm_destroy(ipm_handle* h) {
  if (!h) return IPM_OK;
  cudaSetDevice(h->device);
  if (h->st) cudaStreamSynchronize(h->st);
  free_arena(h);
  if (h->hs) cudaFreeHost(h->hs);
  if (h->st) cudaStreamDestroy(h->st);
  if (h->st2) cudaStreamDestroy(h->st2);
  if (h->st3) cudaStreamDestroy(h->st3);
  if (h->st4) cudaStreamDestroy(h->st4);
  if (h->ev) cudaEventDestroy(h->ev);
  delete h;
  return IPM_OK;
}

// Loads a one-sided QP whose m rows are the m_ar rows of F listed in a_rows followed by the
// m - m_ar rows of the CSR matrix A (either part may be empty); qp->bl is ignored.
static int load_qp(ipm_handle* h, const ipm_qp* qp, int64_t m_ar, void* stream) {
  const int64_t n = qp->n, m = qp->m, fr = qp->f_rows;
  const int mem = qp->mem;
  if (n < 1 || m < 0 || fr < 0 || (mem != IPM_MEM_HOST && mem != IPM_MEM_DEVICE))
    return fail(h, IPM_ERR_ARG, "bad sizes or memory space");
  if (n > INT32_MAX || fr + m > INT32_MAX) return fail(h, IPM_ERR_ARG, "sizes exceed int32 indexing");
  const int64_t m_c = m - m_ar;
  const bool use_arows = m_ar > 0;
  const bool use_acsr = m_c > 0;
  if (m_ar < 0 || m_c < 0 || (use_arows && !qp->a_rows) || (use_acsr && !qp->A_indptr))
    return fail(h, IPM_ERR_ARG, "missing constraint rows");
  if (use_arows && fr == 0) return fail(h, IPM_ERR_ARG, "a_rows needs a factor F");
  int rc;
  HostQP q;
  q.n = n; q.m = m; q.fr = fr;
  // vectors
  if ((rc = fetch(h, qp->c, n, mem, q.c))) return rc;
  if (m && (rc = fetch(h, qp->b, m, mem, q.b))) return rc;
  if (qp->l) { if ((rc = fetch(h, qp->l, n, mem, q.l))) return rc; } else q.l.assign(n, -INFINITY);
  if (qp->u) { if ((rc = fetch(h, qp->u, n, mem, q.u))) return rc; } else q.u.assign(n, INFINITY);
  if (qp->h0) { if ((rc = fetch(h, qp->h0, n, mem, q.h0))) return rc; } else q.h0.assign(n, 0.0);
  for (int64_t j = 0; j < n; ++j) {
    if (!std::isfinite(q.c[j]) || !std::isfinite(q.h0[j]) || q.h0[j] < 0) return fail(h, IPM_ERR_ARG, "c or h0 not finite / h0 < 0");
    if (std::isnan(q.l[j]) || std::isnan(q.u[j]) || q.l[j] == INFINITY || q.u[j] == -INFINITY) return fail(h, IPM_ERR_ARG, "bad bound");
    if (std::isfinite(q.l[j]) && std::isfinite(q.u[j]) && !(q.l[j] < q.u[j])) return fail(h, IPM_ERR_ARG, "l >= u");
  }
  for (int64_t k = 0; k < m; ++k) if (!std::isfinite(q.b[k])) return fail(h, IPM_ERR_ARG, "b not finite");
  // low-rank Hessian term U diag(u_w) U^T
  if (qp->u_cols < 0 || qp->u_cols > (1 << 16)) return fail(h, IPM_ERR_ARG, "u_cols out of range [0, 65536]");
  q.ucols = qp->u_cols;
  if (q.ucols) {
    if (!qp->U || !qp->u_w) return fail(h, IPM_ERR_ARG, "u_cols > 0 needs U and u_w");
    q.U.resize((size_t)(n * q.ucols));
    if ((rc = fetch_into(h, qp->U, n * q.ucols, mem, q.U.data()))) return rc;
    if ((rc = fetch(h, qp->u_w, q.ucols, mem, q.uw))) return rc;
    for (double v : q.uw) if (!std::isfinite(v)) return fail(h, IPM_ERR_ARG, "u_w not finite");
    std::atomic<int> bad{0};
    parallel_ranges((int64_t)q.U.size(), q.U.size() < (1u << 20) ? 1 : host_threads(), [&](int, int64_t b, int64_t e) {
      for (int64_t k = b; k < e; ++k)
        if (!std::isfinite(q.U[k])) { bad.store(1); break; }
    });
    if (bad.load()) return fail(h, IPM_ERR_ARG, "U not finite");
  }
  // R = [F; A_csr], copied straight into the host image of R
  std::vector<int64_t> Fp, Ap;
  std::vector<int32_t> arows_in;
  std::vector<double> fw;
  if (fr) {
    if ((rc = fetch(h, qp->F_indptr, fr + 1, mem, Fp))) return rc;
    if (Fp[0] != 0) return fail(h, IPM_ERR_ARG, "F_indptr[0] != 0");
    for (int64_t r = 0; r < fr; ++r) if (Fp[r + 1] < Fp[r]) return fail(h, IPM_ERR_ARG, "F_indptr not monotone");
    if ((rc = fetch(h, qp->f_w, fr, mem, fw))) return rc;
    for (double w : fw) if (!std::isfinite(w) || w < 0) return fail(h, IPM_ERR_ARG, "f_w must be finite and >= 0");
  }
  if (use_acsr) {
    if ((rc = fetch(h, qp->A_indptr, m_c + 1, mem, Ap))) return rc;
    if (Ap[0] != 0) return fail(h, IPM_ERR_ARG, "A_indptr[0] != 0");
    for (int64_t r = 0; r < m_c; ++r) if (Ap[r + 1] < Ap[r]) return fail(h, IPM_ERR_ARG, "A_indptr not monotone");
  }
  if (use_arows) {
    if ((rc = fetch(h, qp->a_rows, m_ar, mem, arows_in))) return rc;
    std::vector<int32_t> srt(arows_in);
    std::sort(srt.begin(), srt.end());
    for (int64_t k = 0; k < m_ar; ++k) {
      if (srt[k] < 0 || srt[k] >= fr) return fail(h, IPM_ERR_ARG, "a_rows index out of range");
      if (k && srt[k] == srt[k - 1]) return fail(h, IPM_ERR_ARG, "a_rows has duplicates");
    }
  }
  q.nR = fr + m_c;
  const int64_t nnzF = fr ? Fp[fr] : 0, nnzA = use_acsr ? Ap[m_c] : 0;
  q.Rp.resize(q.nR + 1);
  q.wR.assign(q.nR, 0.0);
  for (int64_t r = 0; r <= fr; ++r) q.Rp[r] = fr ? Fp[r] : 0;
  for (int64_t r = 0; r < fr; ++r) q.wR[r] = fw[r];
  for (int64_t k = 1; k <= m_c; ++k) q.Rp[fr + k] = nnzF + Ap[k];
  q.arow.resize(m);
  for (int64_t k = 0; k < m; ++k) q.arow[k] = k < m_ar ? arows_in[k] : (int32_t)(fr + (k - m_ar));
  const int64_t nnzR = nnzF + nnzA;
  // entries of A^T: the constraint rows' lengths
  int64_t nnzAT = 0;
  for (int64_t k = 0; k < m; ++k) nnzAT += q.Rp[q.arow[k] + 1] - q.Rp[q.arow[k]];
  // R^T and A^T are built on the device (transpose.cu) unless options.ingest_host asks for
  // the host transpose; the host path is also the fallback for very long columns
  auto host_transpose = [&]() -> int {
    int rc2;
    q.Ri.resize(nnzR);
    q.Rv.resize(nnzR);
    if (nnzF) {
      if ((rc2 = fetch_into(h, qp->F_indices, nnzF, mem, q.Ri.data()))) return rc2;
      if ((rc2 = fetch_into(h, qp->F_data, nnzF, mem, q.Rv.data()))) return rc2;
    }
    if (nnzA) {
      if ((rc2 = fetch_into(h, qp->A_indices, nnzA, mem, q.Ri.data() + nnzF))) return rc2;
      if ((rc2 = fetch_into(h, qp->A_data, nnzA, mem, q.Rv.data() + nnzF))) return rc2;
    }
    switch (check_csr_entries(nnzR, q.Ri.data(), q.Rv.data(), n)) {
      case 1: return fail(h, IPM_ERR_ARG, "column index out of range");
      case 2: return fail(h, IPM_ERR_ARG, "matrix value not finite");
      default: break;
    }
    // R^T by a stable counting sort (rows increase within each column: deterministic order)
    q.RTp.assign(n + 1, 0);
    q.RTi.resize(nnzR);
    q.RTv.resize(nnzR);
    transpose_csr(q.nR, n, q.Rp.data(), q.Ri.data(), q.Rv.data(), q.RTp.data(), q.RTi.data(), q.RTv.data());
    // A^T: the R^T entries of constraint rows, in R^T's order
    std::vector<unsigned char> is_con(q.nR, 0);
    for (int64_t k = 0; k < m; ++k) is_con[q.arow[k]] = 1;
    q.ATp.assign(n + 1, 0);
    filter_rows(n, q.RTp.data(), q.RTi.data(), q.RTv.data(), is_con.data(), q.ATp.data(), nullptr, nullptr);
    q.ATi.resize(q.ATp[n]);
    q.ATv.resize(q.ATp[n]);
    filter_rows(n, q.RTp.data(), q.RTi.data(), q.RTv.data(), is_con.data(), q.ATp.data(), q.ATi.data(), q.ATv.data());
    return IPM_OK;
  };
  if (nnzF && (!qp->F_indices || !qp->F_data)) return fail(h, IPM_ERR_ARG, "missing F arrays");
  if (nnzA && (!qp->A_indices || !qp->A_data)) return fail(h, IPM_ERR_ARG, "missing A arrays");
  bool host_path = h->opt.ingest_host != 0;
  if (host_path && (rc = host_transpose())) return rc;
  // dense H block -> CSR of its non-zeros (symmetry checked)
  if (qp->H_dense) {
    std::vector<double> Hd;
    if ((rc = fetch(h, qp->H_dense, n * n, mem, Hd))) return rc;
    q.Hp.assign(n + 1, 0);
    double scale = 0;
    for (double v : Hd) { if (!std::isfinite(v)) return fail(h, IPM_ERR_ARG, "H_dense not finite"); scale = std::max(scale, std::fabs(v)); }
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        const double v = Hd[i * n + j];
        if (std::fabs(v - Hd[j * n + i]) > 1e-12 * (1 + scale)) return fail(h, IPM_ERR_ARG, "H_dense not symmetric");
        if (v != 0.0) { q.Hi.push_back((int32_t)j); q.Hv.push_back(v); }
      }
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
      q.Hp[i] = cnt;
      for (int64_t j = 0; j < n; ++j) if (Hd[i * n + j] != 0.0) ++cnt;
    }
    q.Hp[n] = cnt;
  }
  q.fl.resize(n);
  q.fu.resize(n);
  int ncomp = (int)m;
  for (int64_t j = 0; j < n; ++j) {
    q.fl[j] = std::isfinite(q.l[j]) ? 1 : 0;
    q.fu[j] = std::isfinite(q.u[j]) ? 1 : 0;
    ncomp += q.fl[j] + q.fu[j];
  }
  double cn = 0, bn = 0;
  for (double v : q.c) cn = std::max(cn, std::fabs(v));
  for (double v : q.b) bn = std::max(bn, std::fabs(v));
  // stiff-row capacity: the stiff_cap longest constraint rows
  auto store = std::make_shared<MatStore>();
  store->device = h->device;
  store->storage = h->opt.storage;
  {
    std::vector<int64_t> lens(m);
    for (int64_t k = 0; k < m; ++k) lens[k] = q.Rp[q.arow[k] + 1] - q.Rp[q.arow[k]];
    std::sort(lens.begin(), lens.end(), std::greater<int64_t>());
    const int64_t kmax = std::min<int64_t>(m, 1024);
    store->sc_prefix.assign(kmax + 1, 0);
    for (int64_t k = 0; k < kmax; ++k) store->sc_prefix[k + 1] = store->sc_prefix[k] + lens[k];
  }
  int stiff_cap = 1;
  int64_t sc_cap = 1;
  stiff_caps(h->opt, m, store->sc_prefix, &stiff_cap, &sc_cap);
  const bool dense = h->opt.dense_max_n > 0 && n <= h->opt.dense_max_n && h->opt.storage == IPM_STORAGE_F64 &&
                     (h->opt.precond == IPM_PRECOND_DENSE || h->opt.precond == IPM_PRECOND_AUTO);
  // allocate
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  free_arena(h);
  Dev dv{};
  CUDA_TRY(h, cudaDeviceGetAttribute(&dv.sm_count, cudaDevAttrMultiProcessorCount, h->device));
  dv.ucols = q.ucols;
  dv.ucap = std::max<int64_t>(q.ucols, h->opt.u_cap);
  dv.ublocks = (int)std::max<int64_t>(1, std::min<int64_t>(4 * (int64_t)dv.sm_count, n / 32));
  const int64_t nnzHs = (int64_t)q.Hv.size();
  Carver cm(nullptr), cs(nullptr);
  const bool want_df = h->opt.op_arith != IPM_ARITH_F64 && h->opt.storage == IPM_STORAGE_F64;
  carve_matrix(cm, dv, n, m, q.nR, nnzR, nnzAT, nnzHs, h->opt.storage, want_df);
  const int64_t nblk = h->opt.precond == IPM_PRECOND_BLOCK32 ? (n + 31) / 32 : 0;
  carve_state(cs, dv, n, m, q.nR, stiff_cap, sc_cap, dense, h->opt.storage, h->opt.max_ipm, want_df, nblk);
  const size_t mbytes = cm.off + 256, sbytes = cs.off + 256;
  if (h->opt.mem_budget > 0 && (double)(mbytes + sbytes) > h->opt.mem_budget)
    return fail(h, IPM_ERR_OOM, "QP needs " + std::to_string(mbytes + sbytes) + " bytes, over mem_budget");
  if ((rc = dev_alloc(h, &store->ptr, mbytes, "matrices"))) return rc;
  store->bytes = mbytes;
  if ((rc = dev_alloc(h, &h->arena, sbytes, "state"))) return rc;
  h->arena_bytes = sbytes;
  h->mat = store;
  Carver cvm((char*)store->ptr), cvs((char*)h->arena);
  carve_matrix(cvm, dv, n, m, q.nR, nnzR, nnzAT, nnzHs, h->opt.storage, want_df);
  carve_state(cvs, dv, n, m, q.nR, stiff_cap, sc_cap, dense, h->opt.storage, h->opt.max_ipm, want_df, nblk);
  dv.n = n; dv.m = m; dv.nR = q.nR; dv.nnzR = nnzR; dv.nnzHs = nnzHs; dv.nnzA = nnzAT;
  dv.g_rows = heuristic_group(q.nR ? (double)nnzR / (double)q.nR : 0.0);
  dv.g_cols = heuristic_group((double)nnzR / (double)n);
  dv.g_at = heuristic_group((double)nnzAT / (double)n);
  if (h->opt.lanes_rows) dv.g_rows = h->opt.lanes_rows;
  if (h->opt.lanes_cols) dv.g_cols = h->opt.lanes_cols;
  if (h->opt.lanes_at) dv.g_at = h->opt.lanes_at;
  dv.aug = h->opt.system == IPM_SYSTEM_AUGMENTED ? 1 : 0;
  dv.nsys = dv.aug ? n + m : n;
  h->d = dv;
  h->g = make_geo(dv);
  if ((rc = alloc_trace(h))) return rc;
  h->cnorm = cn; h->bnorm = bn; h->ncomp = ncomp; h->sc_cap = sc_cap;
  h->fr = fr;
  if ((rc = enter(h, stream))) return rc;
  auto up = [&](const void* dst, const void* src, size_t nbytes) -> int {
    if (nbytes == 0) return IPM_OK;
    CUDA_TRY(h, cudaMemcpyAsync((void*)dst, src, nbytes, cudaMemcpyHostToDevice, h->st));
    return IPM_OK;
  };
  const Dev& d = h->d;
  if ((rc = up(d.R_ptr, q.Rp.data(), 8 * q.Rp.size()))) return rc;
  if ((rc = up(d.arow, q.arow.data(), 4 * q.arow.size()))) return rc;
  {
    // rows pass order: windows of 1024 consecutive rows (the gathered columns of neighbouring
    // rows overlap), each ordered by row length, longest first (stable), so the row groups
    // sharing a warp run equal trip counts (RT rows pass: 133 -> 129 us; windows of 128
    // gained nothing, one global order 131 us)
    std::vector<int32_t> perm(q.nR);
    order_rows_by_length(q.nR, q.Rp.data(), 1024, perm.data());
    if ((rc = up(d.rperm, perm.data(), 4 * perm.size()))) return rc;
  }
  if (!host_path) {
    // R straight from the caller's arrays (host or device), then R^T and A^T on the device
    auto in = [&](void* dst, const void* src, size_t nbytes) -> int {
      if (nbytes == 0) return IPM_OK;
      CUDA_TRY(h, cudaMemcpyAsync(dst, src, nbytes, cudaMemcpyDefault, h->st));
      return IPM_OK;
    };
    if ((rc = in((void*)d.R_idx, qp->F_indices, 4 * (size_t)nnzF))) return rc;
    if ((rc = in((void*)d.R_val, qp->F_data, 8 * (size_t)nnzF))) return rc;
    if ((rc = in((void*)(d.R_idx + nnzF), qp->A_indices, 4 * (size_t)nnzA))) return rc;
    if ((rc = in((void*)(d.R_val + nnzF), qp->A_data, 8 * (size_t)nnzA))) return rc;
    void* scratch = nullptr;
    if ((rc = dev_alloc(h, &scratch, device_transpose_scratch(n, q.nR), "transpose scratch"))) return rc;
    cudaError_t terr = cudaSuccess;
    const int tr = device_transpose(d.R_ptr, d.R_idx, d.R_val, q.nR, n, nnzR, d.arow, m, (int64_t*)d.RT_ptr,
                                    (int32_t*)d.RT_idx, (double*)d.RT_val, (int64_t*)d.AT_ptr, (int32_t*)d.AT_idx,
                                    (double*)d.AT_val, scratch, dv.sm_count, h->st, &terr);
    cudaStreamSynchronize(h->st);
    cudaFree(scratch);
    if (tr < 0) return fail(h, IPM_ERR_CUDA, std::string("device transpose: ") + cudaGetErrorString(terr));
    if (tr == 1) return fail(h, IPM_ERR_ARG, "column index out of range");
    if (tr == 2) return fail(h, IPM_ERR_ARG, "matrix value not finite");
    if (tr == 3) {
      host_path = true;                 // a column too long for the device sort
      if ((rc = host_transpose())) return rc;
    }
  }
  if (host_path) {
    if ((rc = up(d.R_idx, q.Ri.data(), 4 * q.Ri.size()))) return rc;
    if ((rc = up(d.R_val, q.Rv.data(), 8 * q.Rv.size()))) return rc;
    if ((rc = up(d.RT_ptr, q.RTp.data(), 8 * q.RTp.size()))) return rc;
    if ((rc = up(d.RT_idx, q.RTi.data(), 4 * q.RTi.size()))) return rc;
    if ((rc = up(d.RT_val, q.RTv.data(), 8 * q.RTv.size()))) return rc;
    if ((rc = up(d.AT_ptr, q.ATp.data(), 8 * q.ATp.size()))) return rc;
    if ((rc = up(d.AT_idx, q.ATi.data(), 4 * q.ATi.size()))) return rc;
    if ((rc = up(d.AT_val, q.ATv.data(), 8 * q.ATv.size()))) return rc;
  }
  if (d.Hs_ptr) {
    if ((rc = up(d.Hs_ptr, q.Hp.data(), 8 * q.Hp.size()))) return rc;
    if ((rc = up(d.Hs_idx, q.Hi.data(), 4 * q.Hi.size()))) return rc;
    if ((rc = up(d.Hs_val, q.Hv.data(), 8 * q.Hv.size()))) return rc;
  }
  if (q.ucols) {
    if ((rc = up(d.U, q.U.data(), 8 * q.U.size()))) return rc;
    if ((rc = up(d.uw, q.uw.data(), 8 * q.uw.size()))) return rc;
  }
  if ((rc = up(d.wR, q.wR.data(), 8 * q.wR.size()))) return rc;
  if ((rc = up(d.h0, q.h0.data(), 8 * n))) return rc;
  if ((rc = up(d.c, q.c.data(), 8 * n))) return rc;
  if ((rc = up(d.b, q.b.data(), 8 * m))) return rc;
  if ((rc = up(d.l, q.l.data(), 8 * n))) return rc;
  if ((rc = up(d.u, q.u.data(), 8 * n))) return rc;
  if ((rc = up(d.fl, q.fl.data(), n))) return rc;
  if ((rc = up(d.fu, q.fu.data(), n))) return rc;
  CUDA_TRY(h, cudaMemsetAsync(d.hist, 0, sizeof(unsigned int) * kHistBins, h->st));
  CUDA_TRY(h, cudaMemsetAsync(d.slotR, 0xff, sizeof(int32_t) * std::max<int64_t>(q.nR, 1), h->st));
  CUDA_TRY(h, launch_fill_rowk(d, h->st));
  CUDA_TRY(h, launch_densify_R(d, h->st));
  if (d.ucap) CUDA_TRY(h, cudaMemsetAsync(d.lrs, 0, sizeof(double) * d.ucap, h->st));
  std::memset(h->hs, 0, sizeof(Scal));
  push_options(h);
  h->hs->mu = h->hs->mu0 = 1.0;
  h->hs->status = DS_RUNNING;
  CUDA_TRY(h, cudaMemcpyAsync(d.sc, h->hs, sizeof(Scal), cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, launch_diagH(d, h->st));
  CUDA_TRY(h, launch_quantize(d, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));   // host staging buffers go out of scope
  if ((rc = prepare_operator_formats(h))) return rc;
  if (nblk && (rc = prepare_block_segments(h, q.Rp, q.arow))) return rc;
  if (h->opt.autotune && !h->opt.lanes_rows && !h->opt.lanes_cols && (rc = autotune_groups(h))) return rc;
  h->loaded = true;
  h->have_iterate = false;
  h->precond = choose_precond(h);
  h->info = ipm_info{};
  return leave(h, stream);
}

// Two-sided rows bl <= A x <= b are loaded as the paper's stack B = [A; -A] (Section 4,
// before eq:2x2_reduced): the upper sides A_k x <= b_k (finite b_k), then the lower sides
// -A_k x <= -bl_k (finite bl_k).  Rows of F named by a_rows keep their fused form for the
// upper side; a lower side becomes a negated copy of its row in the explicit CSR block.
int ipm_set_qp(ipm_handle* h, const ipm_qp* qp, void* stream) {
  if (!h || !qp) return IPM_ERR_ARG;
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is in flight on this handle");
  h->err.clear();
  const int64_t m = qp->m, fr = qp->f_rows;
  const int mem = qp->mem;
  if (m < 0 || fr < 0 || (mem != IPM_MEM_HOST && mem != IPM_MEM_DEVICE))
    return fail(h, IPM_ERR_ARG, "bad sizes or memory space");
  const bool use_arows = qp->a_rows != nullptr;
  if (m > 0 && use_arows == (qp->A_indptr != nullptr)) return fail(h, IPM_ERR_ARG, "give exactly one of a_rows or A (CSR)");
  int rc;
  if (!qp->bl || m == 0) {
    if ((rc = load_qp(h, qp, use_arows ? m : 0, stream))) return rc;
    h->m_user = m;
    h->rows_up = m;
    h->stacked = false;
    h->row_of.clear();
    return IPM_OK;
  }
  std::vector<double> b, bl;
  if ((rc = fetch(h, qp->b, m, mem, b)) || (rc = fetch(h, qp->bl, m, mem, bl))) return rc;
  std::vector<int32_t> row_of;
  for (int64_t k = 0; k < m; ++k) {
    if (std::isnan(b[k]) || std::isnan(bl[k]) || b[k] == -INFINITY || bl[k] == INFINITY)
      return fail(h, IPM_ERR_ARG, "b or bl is not a valid row bound");
    // an equality row (bl = b) would drive both sides' slacks to zero together: refused,
    // like l = u for a variable
    if (!(bl[k] < b[k])) return fail(h, IPM_ERR_ARG, "bl >= b");
    if (std::isfinite(b[k])) row_of.push_back((int32_t)k);
  }
  const int64_t up = (int64_t)row_of.size();
  for (int64_t k = 0; k < m; ++k)
    if (std::isfinite(bl[k])) row_of.push_back((int32_t)k);
  const int64_t mr = (int64_t)row_of.size();
  if (fr + mr > INT32_MAX) return fail(h, IPM_ERR_ARG, "sizes exceed int32 indexing");
  std::vector<double> bs(mr);
  for (int64_t r = 0; r < mr; ++r) bs[r] = r < up ? b[row_of[r]] : -bl[row_of[r]];
  // host view of the source rows: F (a_rows) or the caller's A
  const int64_t srows = use_arows ? fr : m;
  std::vector<int64_t> sp;
  std::vector<int32_t> ar, si_h;
  std::vector<double> sv_h;
  if ((rc = fetch(h, use_arows ? qp->F_indptr : qp->A_indptr, srows + 1, mem, sp))) return rc;
  if (sp[0] != 0) return fail(h, IPM_ERR_ARG, "indptr[0] != 0");
  for (int64_t r = 0; r < srows; ++r) if (sp[r + 1] < sp[r]) return fail(h, IPM_ERR_ARG, "indptr not monotone");
  const int32_t* s_idx = use_arows ? qp->F_indices : qp->A_indices;
  const double* s_val = use_arows ? qp->F_data : qp->A_data;
  if (sp[srows] && (!s_idx || !s_val)) return fail(h, IPM_ERR_ARG, "missing matrix arrays");
  const bool need_entries = use_arows ? mr > up : mr > 0;     // rows copied into the CSR block
  if (mem == IPM_MEM_DEVICE && sp[srows] && need_entries) {
    si_h.resize(sp[srows]);
    sv_h.resize(sp[srows]);
    if ((rc = fetch_into(h, s_idx, sp[srows], mem, si_h.data())) || (rc = fetch_into(h, s_val, sp[srows], mem, sv_h.data())))
      return rc;
    s_idx = si_h.data();
    s_val = sv_h.data();
  }
  if (use_arows) {
    if ((rc = fetch(h, qp->a_rows, m, mem, ar))) return rc;
    for (int32_t r : ar) if (r < 0 || r >= fr) return fail(h, IPM_ERR_ARG, "a_rows index out of range");
    std::vector<int32_t> srt(ar);
    std::sort(srt.begin(), srt.end());
    if (std::adjacent_find(srt.begin(), srt.end()) != srt.end()) return fail(h, IPM_ERR_ARG, "a_rows has duplicates");
  }
  // stored rows: a_rows of the upper sides, then the CSR block (negated rows for lower sides)
  std::vector<int32_t> ar_up;
  std::vector<int64_t> Cp(1, 0);
  int64_t cnnz = 0;
  for (int64_t r = 0; r < mr; ++r) {
    const int64_t k = row_of[r];
    if (use_arows && r < up) continue;
    const int64_t src = use_arows ? ar[k] : k;
    cnnz += sp[src + 1] - sp[src];
  }
  std::vector<int32_t> Ci((size_t)cnnz);
  std::vector<double> Cv((size_t)cnnz);
  for (int64_t r = 0, o = 0; r < mr; ++r) {
    const int64_t k = row_of[r];
    if (use_arows && r < up) {
      ar_up.push_back(ar[k]);
      continue;
    }
    const int64_t src = use_arows ? ar[k] : k;
    const double sign = r < up ? 1.0 : -1.0;
    for (int64_t e = sp[src]; e < sp[src + 1]; ++e, ++o) {
      Ci[o] = s_idx[e];
      Cv[o] = sign * s_val[e];
    }
    Cp.push_back(o);
  }
  const int64_t m_ar = (int64_t)ar_up.size(), mc = mr - m_ar;
  ipm_qp q2 = *qp;
  q2.m = mr;
  q2.bl = nullptr;
  q2.b = mr ? bs.data() : nullptr;
  q2.a_rows = m_ar ? ar_up.data() : nullptr;
  q2.A_indptr = mc ? Cp.data() : nullptr;
  q2.A_indices = cnnz ? Ci.data() : nullptr;
  q2.A_data = cnnz ? Cv.data() : nullptr;
  void* tmp = nullptr;
  if (mem == IPM_MEM_DEVICE) {
    // the stacked arrays join the caller's device arrays: one temporary device buffer
    const size_t ob = 0, oa = ob + 8 * (size_t)mr, op = oa + ((4 * (size_t)m_ar + 7) & ~(size_t)7),
                 oi = op + 8 * Cp.size(), ov = oi + ((4 * (size_t)cnnz + 7) & ~(size_t)7), tot = ov + 8 * (size_t)cnnz;
    CUDA_TRY(h, cudaSetDevice(h->device));
    if ((rc = dev_alloc(h, &tmp, tot + 8, "stacked rows"))) return rc;
    char* t = static_cast<char*>(tmp);
    const cudaError_t e = [&]() {
      cudaError_t r = cudaSuccess;
      if (mr && r == cudaSuccess) r = cudaMemcpy(t + ob, bs.data(), 8 * (size_t)mr, cudaMemcpyHostToDevice);
      if (m_ar && r == cudaSuccess) r = cudaMemcpy(t + oa, ar_up.data(), 4 * (size_t)m_ar, cudaMemcpyHostToDevice);
      if (mc && r == cudaSuccess) r = cudaMemcpy(t + op, Cp.data(), 8 * Cp.size(), cudaMemcpyHostToDevice);
      if (cnnz && r == cudaSuccess) r = cudaMemcpy(t + oi, Ci.data(), 4 * (size_t)cnnz, cudaMemcpyHostToDevice);
      if (cnnz && r == cudaSuccess) r = cudaMemcpy(t + ov, Cv.data(), 8 * (size_t)cnnz, cudaMemcpyHostToDevice);
      return r;
    }();
    if (e != cudaSuccess) {
      cudaFree(tmp);
      return fail(h, IPM_ERR_CUDA, std::string("stacked rows upload: ") + cudaGetErrorString(e));
    }
    if (mr) q2.b = reinterpret_cast<const double*>(t + ob);
    if (m_ar) q2.a_rows = reinterpret_cast<const int32_t*>(t + oa);
    if (mc) q2.A_indptr = reinterpret_cast<const int64_t*>(t + op);
    if (cnnz) {
      q2.A_indices = reinterpret_cast<const int32_t*>(t + oi);
      q2.A_data = reinterpret_cast<const double*>(t + ov);
    }
  }
  rc = load_qp(h, &q2, m_ar, stream);
  if (tmp) {
    cudaStreamSynchronize(h->st);
    cudaFree(tmp);
  }
  if (rc) return rc;
  h->m_user = m;
  h->rows_up = up;
  h->stacked = !(up == m && mr == m);          // else one-sided after all: the caller's rows
  if (!h->stacked) row_of.clear();
  h->row_of = std::move(row_of);
  return IPM_OK;
}

int ipm_get_sizes(const ipm_handle* h, int64_t* n, int64_t* m, int64_t* m_rows) {
  if (!h) return IPM_ERR_ARG;
  if (!h->loaded) return IPM_ERR_STATE;
  if (n) *n = h->d.n;
  if (m) *m = h->m_user;
  if (m_rows) *m_rows = h->d.m;
  return IPM_OK;
}

int ipm_share_qp(ipm_handle* h, ipm_handle* src, void* stream) {
  if (!h || !src || h == src) return IPM_ERR_ARG;
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is in flight on this handle");
  if (!src->loaded || !src->mat) return fail(h, IPM_ERR_STATE, "source handle has no QP");
  if (src->device != h->device) return fail(h, IPM_ERR_ARG, "handles on different devices");
  if (src->opt.storage != h->opt.storage) return fail(h, IPM_ERR_ARG, "storage option differs from the source's");
  h->err.clear();
  int rc;
  const Dev& sd = src->d;
  const int64_t n = sd.n, m = sd.m, nR = sd.nR;
  int stiff_cap = 1;
  int64_t sc_cap = 1;
  stiff_caps(h->opt, m, src->mat->sc_prefix, &stiff_cap, &sc_cap);
  const bool use_dense = h->opt.dense_max_n > 0 && n <= h->opt.dense_max_n && h->opt.storage == IPM_STORAGE_F64 &&
                         (h->opt.precond == IPM_PRECOND_DENSE || h->opt.precond == IPM_PRECOND_AUTO);
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  auto store = src->mat;            // keep the matrices alive before dropping our own
  free_arena(h);
  Dev dv = sd;                      // sizes, lane choices and matrix pointers of the source
  Carver cs(nullptr);
  carve_state(cs, dv, n, m, nR, stiff_cap, sc_cap, use_dense, h->opt.storage, h->opt.max_ipm, sd.R_df != nullptr,
              sd.nblk);
  const size_t sbytes = cs.off + 256;
  if (h->opt.mem_budget > 0 && (double)sbytes > h->opt.mem_budget)
    return fail(h, IPM_ERR_OOM, "state needs " + std::to_string(sbytes) + " bytes, over mem_budget");
  if ((rc = dev_alloc(h, &h->arena, sbytes, "state"))) return rc;
  h->arena_bytes = sbytes;
  h->mat = store;
  Carver cvs((char*)h->arena);
  carve_state(cvs, dv, n, m, nR, stiff_cap, sc_cap, use_dense, h->opt.storage, h->opt.max_ipm, sd.R_df != nullptr,
              sd.nblk);
  if (h->opt.lanes_rows) dv.g_rows = h->opt.lanes_rows;
  if (h->opt.lanes_cols) dv.g_cols = h->opt.lanes_cols;
  if (h->opt.lanes_at) dv.g_at = h->opt.lanes_at;
  dv.aug = h->opt.system == IPM_SYSTEM_AUGMENTED ? 1 : 0;
  dv.nsys = dv.aug ? n + m : n;
  h->d = dv;
  h->g = make_geo(dv);
  if ((rc = alloc_trace(h))) return rc;
  h->cnorm = src->cnorm; h->bnorm = src->bnorm; h->ncomp = src->ncomp; h->sc_cap = sc_cap;
  h->fr = src->fr;
  h->stacked = src->stacked;
  h->m_user = src->m_user;
  h->rows_up = src->rows_up;
  h->row_of = src->row_of;
  // the source's problem vectors, ordered after its own stream and the caller's
  CUDA_TRY(h, cudaEventRecord(src->ev, src->st));
  CUDA_TRY(h, cudaStreamWaitEvent(h->st, src->ev, 0));
  if ((rc = enter(h, stream))) return rc;
  const Dev& d = h->d;
  auto cp = [&](const void* dst, const void* from, size_t nbytes) -> int {
    if (nbytes == 0) return IPM_OK;
    CUDA_TRY(h, cudaMemcpyAsync((void*)dst, from, nbytes, cudaMemcpyDeviceToDevice, h->st));
    return IPM_OK;
  };
  if ((rc = cp(d.wR, sd.wR, 8 * nR))) return rc;
  if ((rc = cp(d.h0, sd.h0, 8 * n))) return rc;
  if ((rc = cp(d.c, sd.c, 8 * n))) return rc;
  if ((rc = cp(d.b, sd.b, 8 * m))) return rc;
  if ((rc = cp(d.l, sd.l, 8 * n))) return rc;
  if ((rc = cp(d.u, sd.u, 8 * n))) return rc;
  if ((rc = cp(d.fl, sd.fl, n))) return rc;
  if ((rc = cp(d.fu, sd.fu, n))) return rc;
  if ((rc = cp(d.diagH, sd.diagH, 8 * n))) return rc;
  if (d.ucols && (rc = cp(d.uw, sd.uw, 8 * d.ucols))) return rc;
  if (d.ucols && (rc = cp(d.U, sd.U, 8 * n * d.ucols))) return rc;
  CUDA_TRY(h, cudaMemsetAsync(d.hist, 0, sizeof(unsigned int) * kHistBins, h->st));
  CUDA_TRY(h, cudaMemsetAsync(d.slotR, 0xff, sizeof(int32_t) * std::max<int64_t>(nR, 1), h->st));
  CUDA_TRY(h, launch_fill_rowk(d, h->st));
  CUDA_TRY(h, launch_densify_R(d, h->st));
  if (d.ucap) CUDA_TRY(h, cudaMemsetAsync(d.lrs, 0, sizeof(double) * d.ucap, h->st));
  if (d.nblk) CUDA_TRY(h, launch_block_const(d, h->st));
  std::memset(h->hs, 0, sizeof(Scal));
  push_options(h);
  h->hs->mu = h->hs->mu0 = 1.0;
  h->hs->status = DS_RUNNING;
  CUDA_TRY(h, cudaMemcpyAsync(d.sc, h->hs, sizeof(Scal), cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  h->loaded = true;
  h->have_iterate = false;
  h->precond = choose_precond(h);
  h->info = ipm_info{};
  return leave(h, stream);
}

int ipm_device_bytes(const ipm_handle* h, int64_t* matrix_bytes, int64_t* state_bytes, int* matrix_refs) {
  if (!h) return IPM_ERR_ARG;
  if (matrix_bytes) *matrix_bytes = h->mat ? (int64_t)h->mat->bytes : 0;
  if (state_bytes) *state_bytes = (int64_t)h->arena_bytes;
  if (matrix_refs) *matrix_refs = h->mat ? (int)h->mat.use_count() : 0;
  return IPM_OK;
}

}  // extern "C"

// Launches a whole solve (one graph launch, or the direct-launch loop) and queues the copy
// of the device scalars and trace back to pinned host memory; does not wait.
static int solve_launch(ipm_handle* h, int flags, int64_t* direct_launches) {
  int rc;
  if ((rc = pull_scal(h))) return rc;
  push_options(h);
  h->hs->eta_override = 0;
  h->hs->trace_cap = h->trace_cap;
  CUDA_TRY(h, cudaMemcpyAsync(h->d.sc, h->hs, sizeof(Scal), cudaMemcpyHostToDevice, h->st));
  const bool warm = (flags & IPM_WARM) && h->have_iterate;
  const int pc = h->precond;
  h->have_iterate = true;
  h->pending_pc = pc;
  h->pending_warm = warm;
  if ((rc = ensure_solve_graph(h, pc, warm))) return rc;
  if (h->opt.use_graphs) {
    CUDA_TRY(h, cudaGraphLaunch(h->graphs[pc].solve[warm ? 1 : 0], h->st));
  } else {
    // same kernels launched one by one, loops driven from the host
    const Dev& d = h->d;
    CUDA_TRY(h, warm ? launch_warm_start(d, h->g, h->st) : launch_start_point(d, h->g, h->st));
    CUDA_TRY(h, launch_solve_begin(d, h->st));
    for (int it = 0; it < h->opt.max_ipm; ++it) {
      if ((rc = run_iteration_direct(h, pc, direct_launches))) return rc;
      CUDA_TRY(h, cudaMemcpyAsync(h->hs, d.sc, sizeof(Scal), cudaMemcpyDeviceToHost, h->st));
      CUDA_TRY(h, cudaStreamSynchronize(h->st));
      if (h->hs->stop) break;
    }
  }
  CUDA_TRY(h, cudaMemcpyAsync(h->hs, h->d.sc, sizeof(Scal), cudaMemcpyDeviceToHost, h->st));
  if (h->trace_cap)
    CUDA_TRY(h, cudaMemcpyAsync(h->htrace, h->d.trace, sizeof(double) * kTraceCols * (size_t)h->trace_cap,
                                cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaEventRecord(h->ev, h->st));
  h->pending = 1;
  return IPM_OK;
}

static int fill_info(ipm_handle* h, int64_t direct_launches);

// Waits for the launched solve (bounded by timeout_ms) and fills h->info and h->trace.
static int solve_collect(ipm_handle* h, int64_t direct_launches) {
  const auto t0 = h->t_launch;
  if (h->opt.timeout_ms > 0) {
    while (true) {
      cudaError_t q = cudaEventQuery(h->ev);
      if (q == cudaSuccess) break;
      if (q != cudaErrorNotReady) return fail(h, IPM_ERR_CUDA, cudaGetErrorString(q));
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (ms > h->opt.timeout_ms) {
        h->info.status = IPM_ERR_TIMEOUT;
        return fail(h, IPM_ERR_TIMEOUT, "timeout_ms exceeded (the solve keeps running to its iteration limit)");
      }
      std::this_thread::yield();
    }
  } else {
    CUDA_TRY(h, cudaEventSynchronize(h->ev));
  }
  return fill_info(h, direct_launches);
}

// Result bookkeeping after a finished solve: info from the pinned scalars and trace rows.
static int fill_info(ipm_handle* h, int64_t direct_launches) {
  const auto t0 = h->t_launch;
  h->pending = 0;
  const Scal& s = *h->hs;
  const int pc = h->pending_pc;
  const LoopCounts& lc = h->graphs[pc].solve_c[h->pending_warm ? 1 : 0];
  const int rows = std::min(s.trace_rows, h->trace_cap);
  h->trace.assign(h->htrace, h->htrace + (size_t)rows * kTraceCols);
  int64_t launches = direct_launches;
  if (h->opt.use_graphs) {
    launches = lc.top;
    const bool lowp = h->d.storage != ST_F64;
    for (int r = 0; r < rows; ++r) {
      const double* t = h->htrace + (size_t)r * kTraceCols;
      const int64_t cg = (int64_t)t[8], ref = (int64_t)t[13];
      launches += lc.ipm + 1;  // + the loop re-arm kernel counted in ipm
      if (!lowp) {
        launches += std::max<int64_t>(1, cg) * lc.pcg;
      } else if (lc.ru) {
        launches += std::max<int64_t>(1, cg) * lc.pcg + lc.fallback;
      } else {
        launches += (cg + ref) * lc.pcg + ref * lc.refine + lc.fallback;
      }
    }
  }
  int status = s.status == DS_OK ? IPM_OK : s.status == DS_MAX_ITER ? IPM_MAX_ITER
             : s.status == DS_CG_STALL ? IPM_CG_STALL : s.status == DS_RUNNING ? IPM_MAX_ITER
             : s.status == DS_TIMEOUT ? IPM_ERR_TIMEOUT : s.status == DS_INFEASIBLE ? IPM_INFEASIBLE_SUSPECTED
             : IPM_NUMERICAL;
  ipm_info& in = h->info;
  in.status = status;
  in.ipm_iters = s.ipm_iter;
  in.cg_iters = s.cg_total;
  in.max_cg_step = s.max_cg_step;
  in.max_stiff_rows = s.max_stiff_seen;
  in.precond = pc == PC_BLOCK32 ? IPM_PRECOND_BLOCK32 : pc;
  in.rel_kkt = s.rel_kkt;
  in.primal_res = s.res_primal;
  in.dual_res = s.res_dual;
  in.gap_res = s.res_gap;
  in.primal_obj = s.pobj;
  in.dual_obj = s.dobj;
  in.mu = s.mu;
  in.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  in.kernel_launches = launches;
  in.lanes_rows = h->d.g_rows;
  in.lanes_cols = h->d.g_cols;
  in.refine_passes = h->d.storage != ST_F64 ? s.refine_total : 0;
  in.fallback_steps = h->d.storage != ST_F64 ? s.fallback_total : 0;
  in.op_arith = h->d.mx ? IPM_ARITH_MIXED : h->d.df ? IPM_ARITH_DF32 : IPM_ARITH_F64;
  in.rows_runs = h->d.runs;
  in.cols_gap = h->d.gap;
  return status;
}

extern "C" {

int ipm_solve_async(ipm_handle* h, void* stream, int flags) {
  if (!h) return IPM_ERR_ARG;
  if (!h->loaded) return fail(h, IPM_ERR_STATE, "ipm_solve before ipm_set_qp");
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is already in flight on this handle");
  if (!h->opt.use_graphs) return fail(h, IPM_ERR_STATE, "asynchronous solves need use_graphs = 1");
  h->err.clear();
  int rc;
  h->t_launch = std::chrono::steady_clock::now();
  if ((rc = enter(h, stream))) return rc;
  int64_t dl = 0;
  if ((rc = solve_launch(h, flags, &dl))) return rc;
  return leave(h, stream);
}

int ipm_solve_wait(ipm_handle* h, ipm_info* info) {
  if (!h) return IPM_ERR_ARG;
  if (!h->pending) return fail(h, IPM_ERR_STATE, "no solve in flight");
  int st = solve_collect(h, 0);
  if (info) *info = h->info;
  return st;
}

int ipm_solve_query(ipm_handle* h) {
  if (!h) return IPM_ERR_ARG;
  if (!h->pending) return IPM_OK;
  cudaError_t q = cudaEventQuery(h->ev);
  if (q == cudaErrorNotReady) return IPM_BUSY;
  if (q != cudaSuccess) return fail(h, IPM_ERR_CUDA, cudaGetErrorString(q));
  return IPM_OK;
}

int ipm_solve(ipm_handle* h, void* stream, int flags) {
  if (!h) return IPM_ERR_ARG;
  if (!h->loaded) return fail(h, IPM_ERR_STATE, "ipm_solve before ipm_set_qp");
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is already in flight on this handle");
  h->err.clear();
  int rc;
  h->t_launch = std::chrono::steady_clock::now();
  if ((rc = enter(h, stream))) return rc;
  int64_t dl = 0;
  if ((rc = solve_launch(h, flags, &dl))) return rc;
  const int st = solve_collect(h, dl);
  if (st == IPM_ERR_TIMEOUT || st == IPM_ERR_CUDA) return st;
  if ((rc = leave(h, stream))) return rc;
  return st;
}

int ipm_get_info(ipm_handle* h, ipm_info* info) {
  if (!h || !info) return IPM_ERR_ARG;
  if (!h->loaded) return fail(h, IPM_ERR_STATE, "no QP loaded");
  // the operator's configuration is known from ipm_set_qp on, solved or not
  h->info.op_arith = h->d.mx ? IPM_ARITH_MIXED : h->d.df ? IPM_ARITH_DF32 : IPM_ARITH_F64;
  h->info.rows_runs = h->d.runs;
  h->info.cols_gap = h->d.gap;
  h->info.lanes_rows = h->d.g_rows;
  h->info.lanes_cols = h->d.g_cols;
  *info = h->info;
  return IPM_OK;
}

int ipm_get_xyz(ipm_handle* h, double* x, double* y, double* zl, double* zu, double* s, ipm_info* info, int mem, void* stream) {
  if (!h) return IPM_ERR_ARG;
  if (!h->loaded || !h->have_iterate) return fail(h, IPM_ERR_STATE, "no iterate");
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is in flight on this handle (collect it with ipm_solve_wait)");
  int rc;
  if ((rc = enter(h, stream))) return rc;
  const Dev& d = h->d;
  if ((rc = copy_out(h, x, d.x, d.n, mem))) return rc;
  if ((rc = copy_out(h, zl, d.zl, d.n, mem))) return rc;
  if ((rc = copy_out(h, zu, d.zu, d.n, mem))) return rc;
  if (!h->stacked) {
    if ((rc = copy_out(h, y, d.y, d.m, mem))) return rc;
    if ((rc = copy_out(h, s, d.s, d.m, mem))) return rc;
  } else if (y || s) {
    // stored rows -> caller rows: y_k = y_upper - y_lower; s_k = the upper slack, else the lower
    const int64_t mr = d.m, mu = h->m_user;
    std::vector<double> yi(mr), si(mr), yo(mu, 0.0), so(mu, INFINITY);
    if (mr) {
      CUDA_TRY(h, cudaMemcpyAsync(yi.data(), d.y, 8 * (size_t)mr, cudaMemcpyDeviceToHost, h->st));
      CUDA_TRY(h, cudaMemcpyAsync(si.data(), d.s, 8 * (size_t)mr, cudaMemcpyDeviceToHost, h->st));
      CUDA_TRY(h, cudaStreamSynchronize(h->st));
    }
    for (int64_t r = 0; r < mr; ++r) {
      const int32_t k = h->row_of[r];
      if (r < h->rows_up) {
        yo[k] += yi[r];
        so[k] = si[r];
      } else {
        yo[k] -= yi[r];
        if (so[k] == INFINITY) so[k] = si[r];
      }
    }
    if (y && mu) CUDA_TRY(h, cudaMemcpyAsync(y, yo.data(), 8 * (size_t)mu, cudaMemcpyDefault, h->st));
    if (s && mu) CUDA_TRY(h, cudaMemcpyAsync(s, so.data(), 8 * (size_t)mu, cudaMemcpyDefault, h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));   // yo, so go out of scope
  }
  if (mem == IPM_MEM_HOST) CUDA_TRY(h, cudaStreamSynchronize(h->st));
  if (info) ipm_get_info(h, info);
  return leave(h, stream);
}

int ipm_set_iterate(ipm_handle* h, const double* x, const double* s, const double* y, const double* zl,
                    const double* zu, double mu, int mem, void* stream) {
  if (!h) return IPM_ERR_ARG;
  if (!h->loaded) return fail(h, IPM_ERR_STATE, "ipm_set_iterate before ipm_set_qp");
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is in flight on this handle (collect it with ipm_solve_wait)");
  if (!(mu > 0) || !std::isfinite(mu)) return fail(h, IPM_ERR_ARG, "mu must be positive");
  int rc;
  const Dev& d = h->d;
  // validate strict interiority on a host copy
  std::vector<double> hx, hs_, hy, hzl, hzu, hl(d.n), hu(d.n);
  if ((rc = fetch(h, x, d.n, mem, hx)) || (rc = fetch(h, s, d.m, mem, hs_)) || (rc = fetch(h, y, d.m, mem, hy)) ||
      (rc = fetch(h, zl, d.n, mem, hzl)) || (rc = fetch(h, zu, d.n, mem, hzu)))
    return rc;
  CUDA_TRY(h, cudaMemcpy(hl.data(), d.l, 8 * d.n, cudaMemcpyDeviceToHost));
  CUDA_TRY(h, cudaMemcpy(hu.data(), d.u, 8 * d.n, cudaMemcpyDeviceToHost));
  for (int64_t j = 0; j < d.n; ++j) {
    if (!std::isfinite(hx[j])) return fail(h, IPM_ERR_ARG, "x not finite");
    if (std::isfinite(hl[j]) && !(hx[j] > hl[j] && hzl[j] > 0)) return fail(h, IPM_ERR_ARG, "x/z_l not interior");
    if (std::isfinite(hu[j]) && !(hx[j] < hu[j] && hzu[j] > 0)) return fail(h, IPM_ERR_ARG, "x/z_u not interior");
    if (!std::isfinite(hl[j])) hzl[j] = 0.0;
    if (!std::isfinite(hu[j])) hzu[j] = 0.0;
  }
  for (int64_t k = 0; k < d.m; ++k)
    if (!(hs_[k] > 0 && hy[k] > 0) || !std::isfinite(hs_[k]) || !std::isfinite(hy[k])) return fail(h, IPM_ERR_ARG, "s/y not positive");
  if ((rc = enter(h, stream))) return rc;
  if ((rc = copy_in(h, d.x, hx.data(), d.n, IPM_MEM_HOST))) return rc;
  if ((rc = copy_in(h, d.s, hs_.data(), d.m, IPM_MEM_HOST))) return rc;
  if ((rc = copy_in(h, d.y, hy.data(), d.m, IPM_MEM_HOST))) return rc;
  if ((rc = copy_in(h, d.zl, hzl.data(), d.n, IPM_MEM_HOST))) return rc;
  if ((rc = copy_in(h, d.zu, hzu.data(), d.n, IPM_MEM_HOST))) return rc;
  if ((rc = pull_scal(h))) return rc;
  push_options(h);
  h->hs->mu = mu;
  h->hs->mu0 = mu;
  h->hs->status = DS_RUNNING;
  h->hs->stop = 0;
  CUDA_TRY(h, cudaMemcpyAsync(d.sc, h->hs, sizeof(Scal), cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, launch_residual_summary(d, h->g, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  h->have_iterate = true;
  return leave(h, stream);
}

int ipm_residuals(ipm_handle* h, double* rd, double* rp, double* rs, double* rl, double* ru, double* kkt, int mem, void* stream) {
  if (!h) return IPM_ERR_ARG;
  if (!h->loaded || !h->have_iterate) return fail(h, IPM_ERR_STATE, "no iterate");
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is in flight on this handle (collect it with ipm_solve_wait)");
  int rc;
  if ((rc = enter(h, stream))) return rc;
  const Dev& d = h->d;
  CUDA_TRY(h, launch_residual_summary(d, h->g, h->st));
  // complementarity residuals into scratch vectors (ds: r_s, dzl: r_l, dzu: r_u)
  CUDA_TRY(h, launch_comp_resid(d, h->g, h->st));
  if ((rc = copy_out(h, rd, d.rd, d.n, mem))) return rc;
  if ((rc = copy_out(h, rp, d.rp, d.m, mem))) return rc;
  if ((rc = copy_out(h, rs, d.ds, d.m, mem))) return rc;
  if ((rc = copy_out(h, rl, d.dzl, d.n, mem))) return rc;
  if ((rc = copy_out(h, ru, d.dzu, d.n, mem))) return rc;
  if ((rc = pull_scal(h))) return rc;
  if (kkt) {
    kkt[0] = h->hs->rel_kkt;
    kkt[1] = h->hs->res_primal;
    kkt[2] = h->hs->res_dual;
    kkt[3] = h->hs->res_gap;
  }
  return leave(h, stream);
}

int ipm_apply_kkt(ipm_handle* h, const double* p, double* q, int mem, void* stream) {
  if (!h || !p || !q) return IPM_ERR_ARG;
  if (!h->loaded || !h->have_iterate) return fail(h, IPM_ERR_STATE, "no iterate");
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is in flight on this handle (collect it with ipm_solve_wait)");
  int rc;
  if ((rc = enter(h, stream))) return rc;
  const Dev& d = h->d;
  CUDA_TRY(h, launch_diag_update(d, h->g, h->st));
  if ((rc = copy_in(h, d.p, p, d.n, mem))) return rc;
  CUDA_TRY(h, launch_apply(d, h->g, h->st));
  if ((rc = copy_out(h, q, d.q, d.n, mem))) return rc;
  if (mem == IPM_MEM_HOST) CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return leave(h, stream);
}

int ipm_precond_diag(ipm_handle* h, double* diag, int mem, void* stream) {
  if (!h || !diag) return IPM_ERR_ARG;
  if (!h->loaded || !h->have_iterate) return fail(h, IPM_ERR_STATE, "no iterate");
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is in flight on this handle (collect it with ipm_solve_wait)");
  int rc;
  if ((rc = enter(h, stream))) return rc;
  const Dev& d = h->d;
  CUDA_TRY(h, launch_diag_update(d, h->g, h->st));
  CUDA_TRY(h, launch_jacobi_full(d, h->g, d.q, h->st));
  if ((rc = copy_out(h, diag, d.q, d.n, mem))) return rc;
  if (mem == IPM_MEM_HOST) CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return leave(h, stream);
}

int ipm_newton_direction(ipm_handle* h, double eta, double* dx, double* ds, double* dy, double* dzl, double* dzu,
                         ipm_cg_report* rep, int mem, void* stream) {
  if (!h) return IPM_ERR_ARG;
  if (!h->loaded || !h->have_iterate) return fail(h, IPM_ERR_STATE, "no iterate");
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is in flight on this handle (collect it with ipm_solve_wait)");
  int rc;
  if ((rc = enter(h, stream))) return rc;
  const Dev& d = h->d;
  // residual summary at the current iterate, then eta
  CUDA_TRY(h, launch_residual_summary(d, h->g, h->st));
  if ((rc = pull_scal(h))) return rc;
  push_options(h);
  Scal& s = *h->hs;
  if (eta > 0) {
    s.eta = eta;
  } else {
    double e = s.eta_factor * s.rel_kkt;
    s.eta = std::min(s.eta_max, std::max(s.eta_min, std::isfinite(e) ? e : s.eta_max));
  }
  CUDA_TRY(h, cudaMemcpyAsync(d.sc, h->hs, sizeof(Scal), cudaMemcpyHostToDevice, h->st));
  if ((rc = ensure_dir_graph(h, h->precond))) return rc;
  CUDA_TRY(h, cudaGraphLaunch(h->graphs[h->precond].dir, h->st));
  if ((rc = copy_out(h, dx, d.dx, d.n, mem))) return rc;
  if ((rc = copy_out(h, ds, d.ds, d.m, mem))) return rc;
  if ((rc = copy_out(h, dy, d.dy, d.m, mem))) return rc;
  if ((rc = copy_out(h, dzl, d.dzl, d.n, mem))) return rc;
  if ((rc = copy_out(h, dzu, d.dzu, d.n, mem))) return rc;
  if ((rc = pull_scal(h))) return rc;
  if (rep) {
    rep->iters = s.cg_iter;
    rep->converged = s.cg_conv;
    rep->stiff_rows = h->precond == PC_JACOBI_LR ? s.n_stiff : 0;
    rep->rel_res = s.rhs2 > 0 ? std::sqrt(s.rr / s.rhs2) : 0.0;
    rep->eta = s.eta;
  }
  return leave(h, stream);
}

int ipm_step_lengths(ipm_handle* h, const double* dx, const double* ds, const double* dy, const double* dzl,
                     const double* dzu, double tau, double* alpha_p, double* alpha_d, int mem, void* stream) {
  if (!h || !alpha_p || !alpha_d) return IPM_ERR_ARG;
  if (!h->loaded || !h->have_iterate) return fail(h, IPM_ERR_STATE, "no iterate");
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is in flight on this handle (collect it with ipm_solve_wait)");
  if (!(tau > 0 && tau <= 1)) return fail(h, IPM_ERR_ARG, "tau must be in (0, 1]");
  int rc;
  if ((rc = enter(h, stream))) return rc;
  const Dev& d = h->d;
  if ((rc = copy_in(h, d.dx, dx, d.n, mem))) return rc;
  if ((rc = copy_in(h, d.ds, ds, d.m, mem))) return rc;
  if ((rc = copy_in(h, d.dy, dy, d.m, mem))) return rc;
  if ((rc = copy_in(h, d.dzl, dzl, d.n, mem))) return rc;
  if ((rc = copy_in(h, d.dzu, dzu, d.n, mem))) return rc;
  if ((rc = pull_scal(h))) return rc;
  const double tau_keep = h->hs->tau;
  const int eq_keep = h->hs->equal_steps;
  if ((rc = set_scal_double(h, &d.sc->tau, tau))) return rc;
  int zero = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&d.sc->equal_steps, &zero, sizeof(int), cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, launch_ratio(d, h->g, h->st));
  if ((rc = pull_scal(h))) return rc;
  *alpha_p = h->hs->alpha_p;
  *alpha_d = h->hs->alpha_d;
  if ((rc = set_scal_double(h, &d.sc->tau, tau_keep))) return rc;
  CUDA_TRY(h, cudaMemcpyAsync(&d.sc->equal_steps, &eq_keep, sizeof(int), cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return leave(h, stream);
}

}  // extern "C"

struct ipm_batch {
  std::vector<ipm_handle*> hs;
  std::vector<uint64_t> gens;       // each member's ipm_handle::gen when the graph was captured
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr, fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t exec = nullptr;
};

static void batch_free(ipm_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto e : b->join) if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

extern "C" {

int ipm_batch_create(ipm_handle* const* handles, int count, int flags, ipm_batch** out) {
  if (!handles || count < 1 || !out || flags != IPM_COLD) return IPM_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!handles[i] || !handles[i]->loaded || handles[i]->pending || !handles[i]->opt.use_graphs) return IPM_ERR_STATE;
    if (handles[i]->device != handles[0]->device) return IPM_ERR_ARG;
    for (int j = 0; j < i; ++j) if (handles[j] == handles[i]) return IPM_ERR_ARG;
  }
  ipm_batch* b = new (std::nothrow) ipm_batch();
  if (!b) return IPM_ERR_OOM;
  b->hs.assign(handles, handles + count);
  for (int i = 0; i < count; ++i) b->gens.push_back(handles[i]->gen);
  b->join.assign(count, nullptr);
  auto bad = [&](ipm_handle* h, const std::string& m) {
    if (h) h->err = m;
    cudaGetLastError();
    batch_free(b);
    return IPM_ERR_CUDA;
  };
  if (cudaSetDevice(handles[0]->device) != cudaSuccess || cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    return bad(handles[0], "batch stream/event");
  for (auto& e : b->join)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return bad(handles[0], "batch event");
  cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->st);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    ipm_handle* h = b->hs[i];
    const int pc = h->precond;
    Graphs& gr = h->graphs[pc];
    e = cudaStreamWaitEvent(h->st, b->fork, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d.sc, h->hs, sizeof(Scal), cudaMemcpyHostToDevice, h->st);
    gr.solve_c[0] = LoopCounts{};
    if (e == cudaSuccess) e = emit_solve(h, pc, false, h->st, &gr.solve_c[0]);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->hs, h->d.sc, sizeof(Scal), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess && h->trace_cap)
      e = cudaMemcpyAsync(h->htrace, h->d.trace, sizeof(double) * kTraceCols * (size_t)h->trace_cap,
                          cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaEventRecord(b->join[i], h->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->join[i], 0);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->st, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bad(handles[0], std::string("batch capture: ") + cudaGetErrorString(e));
  *out = b;
  return IPM_OK;
}

int ipm_batch_solve(ipm_batch* b, void* stream, int* statuses) {
  if (!b) return IPM_ERR_ARG;
  ipm_handle* h0 = b->hs[0];
  if (cudaSetDevice(h0->device) != cudaSuccess) return IPM_ERR_CUDA;
  const auto t0 = std::chrono::steady_clock::now();
  for (size_t i = 0; i < b->hs.size(); ++i) {
    ipm_handle* h = b->hs[i];
    if (h->pending || !h->loaded) return fail(h, IPM_ERR_STATE, "batch member busy or without a QP");
    // the captured graph holds this member's buffers and kernel parameters as they were at
    // ipm_batch_create; after a reload, ipm_share_qp or ipm_set_lowrank they are gone or stale
    if (h->gen != b->gens[i])
      return fail(h, IPM_ERR_STATE, "batch member changed since ipm_batch_create (create the batch again)");
  }
  for (ipm_handle* h : b->hs) {
    push_options(h);
    h->hs->eta_override = 0;
    h->hs->trace_cap = h->trace_cap;
  }
  if (cudaEventRecord(b->ev, (cudaStream_t)stream) != cudaSuccess || cudaStreamWaitEvent(b->st, b->ev, 0) != cudaSuccess ||
      cudaGraphLaunch(b->exec, b->st) != cudaSuccess || cudaEventRecord(b->ev, b->st) != cudaSuccess ||
      cudaEventSynchronize(b->ev) != cudaSuccess) {
    cudaGetLastError();
    return fail(h0, IPM_ERR_CUDA, "batch launch failed");
  }
  int worst = IPM_OK;
  for (size_t i = 0; i < b->hs.size(); ++i) {
    ipm_handle* h = b->hs[i];
    h->have_iterate = true;
    h->pending_pc = h->precond;
    h->pending_warm = 0;
    h->t_launch = t0;
    const int st = fill_info(h, 0);
    if (statuses) statuses[i] = st;
    if (st != IPM_OK && worst == IPM_OK) worst = st;
  }
  if (cudaStreamWaitEvent((cudaStream_t)stream, b->ev, 0) != cudaSuccess) return IPM_ERR_CUDA;
  return worst;
}

int ipm_batch_destroy(ipm_batch* b) {
  if (!b) return IPM_OK;
  if (b->st) cudaStreamSynchronize(b->st);
  batch_free(b);
  return IPM_OK;
}

int ipm_get_trace(const ipm_handle* h, double* buf, int max_rows) {
  if (!h) return 0;
  const int rows = (int)(h->trace.size() / IPM_TRACE_COLS);
  if (buf && max_rows > 0)
    std::memcpy(buf, h->trace.data(), sizeof(double) * IPM_TRACE_COLS * (size_t)std::min(rows, max_rows));
  return rows;
}

int ipm_profile_operator(ipm_handle* h, int reps, double* ms_rows, double* ms_cols, double* bytes_rows,
                         double* bytes_cols, double* flops_rows, double* flops_cols) {
  if (!h || reps < 1) return IPM_ERR_ARG;
  if (!h->loaded || !h->have_iterate) return fail(h, IPM_ERR_STATE, "no iterate");
  if (h->pending) return fail(h, IPM_ERR_STATE, "a solve is in flight on this handle (collect it with ipm_solve_wait)");
  CUDA_TRY(h, cudaSetDevice(h->device));
  const Dev& d = h->d;
  const Geo& g = h->g;
  CUDA_TRY(h, launch_diag_update(d, g, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(d.p, d.x, sizeof(double) * d.n, cudaMemcpyDeviceToDevice, h->st));
  // the passes the handle's PCG runs: FP64, or the reduced-precision ones of its storage
  const bool lp = d.storage != ST_F64;
  if (lp) CUDA_TRY(h, launch_mirror_p32(d, g, h->st));
  if (d.df || d.mx) CUDA_TRY(h, launch_mirror_df(d, g, h->st));
  auto rows = [&]() {
    cudaError_t e = lp ? launch_op_rows_lp_only(d, g, h->st) : launch_op_rows_only(d, g, h->st);
    if (e == cudaSuccess && d.ucols) e = launch_lr(d, d.p, 0, h->st);   // U^T p belongs to the first half
    return e;
  };
  auto cols = [&]() { return lp ? launch_op_cols_lp_only(d, g, h->st) : launch_op_cols_only(d, g, h->st); };
  std::vector<cudaEvent_t> ev(3 * reps);
  for (auto& e : ev) CUDA_TRY(h, cudaEventCreate(&e));
  // one untimed pair first
  CUDA_TRY(h, rows());
  CUDA_TRY(h, cols());
  for (int r = 0; r < reps; ++r) {
    CUDA_TRY(h, cudaEventRecord(ev[3 * r], h->st));
    CUDA_TRY(h, rows());
    CUDA_TRY(h, cudaEventRecord(ev[3 * r + 1], h->st));
    CUDA_TRY(h, cols());
    CUDA_TRY(h, cudaEventRecord(ev[3 * r + 2], h->st));
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  double tr = 0, tc = 0;
  for (int r = 0; r < reps; ++r) {
    float a = 0, b = 0;
    CUDA_TRY(h, cudaEventElapsedTime(&a, ev[3 * r], ev[3 * r + 1]));
    CUDA_TRY(h, cudaEventElapsedTime(&b, ev[3 * r + 1], ev[3 * r + 2]));
    tr += a;
    tc += b;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  const double nnz = (double)d.nnzR, nnzh = (double)d.nnzHs, nR = (double)d.nR, n = (double)d.n;
  if (ms_rows) *ms_rows = tr / reps;
  if (ms_cols) *ms_cols = tc / reps;
  // low-rank term: U read once in each half (U^T p, then U (W t)), p and W t read once
  const double lr_b = d.ucols ? 8.0 * n * (double)d.ucols + 8.0 * (double)d.ucols : 0.0;
  const double lr_f = d.ucols ? 2.0 * n * (double)d.ucols : 0.0;
  // the rows pass reads, per row, its row pointers (CSR) or its run pointers and runs
  // (pieces: the row pointers of R for the entry offsets, the piece pointers, 8 bytes a piece)
  const double row_index = d.runs ? 16.0 * (nR + 1) + 8.0 * (double)d.npieces : 4.0 * nnz + 8.0 * (nR + 1);
  const double hs_b = d.Hs_ptr ? 12.0 * nnzh + 8.0 * (n + 1) : 0.0;
  if (lp) {
    const double vb = d.storage == ST_F32 ? 4.0 : (d.storage == ST_BF16 ? 2.0 : 1.0);
    // rows: narrow values, the index data, scale, w_R, thR read, w32 written, p32 read once
    if (bytes_rows) *bytes_rows = vb * nnz + row_index + 24.0 * nR + 4.0 * n + lr_b;
    // cols: narrow values + indices (CSR: 4 bytes an entry; gap layout: 2 bytes a slot and a base
    // row per column), column pointers, w32 read once, p, h0, sigma read, q written
    const double col_data = d.gap ? (vb + 2.0) * (double)d.nslots + 4.0 * n : (vb + 4.0) * nnz;
    if (bytes_cols) *bytes_cols = col_data + 8.0 * (n + 1) + 4.0 * nR + 32.0 * n + hs_b + lr_b;
    if (flops_rows) *flops_rows = 2.0 * nnz + 4.0 * nR + lr_f;
    if (flops_cols) *flops_cols = 2.0 * nnz + 2.0 * nnzh + 4.0 * n + lr_f;
    return IPM_OK;
  }
  // FP64 and double-float alike (8 bytes per value and per vector entry):
  // rows: values, the index data, the row order, omega, v written, p read once
  if (bytes_rows) *bytes_rows = 8.0 * nnz + row_index + 4.0 * nR + 16.0 * nR + 8.0 * n + lr_b;
  // cols: values + indices, row pointers, v read once, p, h0, sigma read, q written (+ Hs)
  if (bytes_cols) *bytes_cols = 12.0 * nnz + 8.0 * (n + 1) + 8.0 * nR + 32.0 * n + hs_b + lr_b;
  if (flops_rows) *flops_rows = 2.0 * nnz + nR + lr_f;
  if (flops_cols) *flops_cols = 2.0 * nnz + 2.0 * nnzh + 4.0 * n + lr_f;
  return IPM_OK;
}

}  // extern "C"
