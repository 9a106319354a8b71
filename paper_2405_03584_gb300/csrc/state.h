// Device pointer bundle of one solver handle and the host-side launch interface of the kernels.
// Every kernel takes the bundle by value; sizes are fixed per loaded QP, so a captured CUDA
// graph stays valid until the next ipm_set_qp.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ipmk {

constexpr int kTraceCols = 14;   // columns of one trace row (IPM_TRACE_COLS of the C header)

struct Dev {
  int64_t n, m, nR;            // variables, constraint rows, rows of R = [F; A_csr]
  int64_t nsys;                // PCG unknowns: n (condensed system), n + m (doubly augmented)
  int aug;                     // 1: PCG on the doubly augmented system (Section 4, eq:2x2_augmented)
  int64_t nnzR, nnzHs;
  int g_rows, g_cols;          // lanes per row of the kernels over R and over R^T (4, 8, 16, 32)
  int g_at;                    // lanes per row of the kernels over A^T alone
  int sm_count;                // multiprocessors of the device (grid sizing)
  // problem data
  const int64_t* R_ptr; const int32_t* R_idx; const double* R_val;
  const int64_t* RT_ptr; const int32_t* RT_idx; const double* RT_val;
  // A^T alone: the entries of R^T whose row is a constraint row (same row indices, same order)
  const int64_t* AT_ptr; const int32_t* AT_idx; const double* AT_val;
  int64_t nnzA;
  const int64_t* Hs_ptr; const int32_t* Hs_idx; const double* Hs_val;   // nullptr if none
  const int32_t* arow;         // m: row of R holding constraint k
  const int32_t* rperm;        // nR: order of the rows in the PCG rows pass (nullptr: natural)
  // low-rank Hessian term U diag(uw) U^T (eq:bfgs_hessian): U is n x ucols, row-major
  int64_t ucols;               // columns in use (<= ucap); U's row stride
  int64_t ucap;                // columns allocated (per handle: U is part of the state)
  double* U;
  double* uw;                  // ucols weights
  double* lrs;                 // ucols: uw o (U^T v) for the vector v of the last launch_lr
  double* upart;               // ublocks x ucols partial sums of U^T v
  double* lrq;                 // ucols: uw o t^2 (terms of v^T U W U^T v)
  int ublocks;
  const double *wR, *h0, *c, *b, *l, *u;
  const unsigned char *fl, *fu;  // finite-bound masks (n)
  double* diagH;               // n: diag(H), computed once
  // iterate
  double *x, *s, *y, *zl, *zu;
  // per IPM iteration
  double *theta, *sigma, *omega, *M0, *Minv, *thR;  // thR: theta placed on R rows (Jacobi part)
  double *rd, *rp, *Hx, *Aty;
  double *tR, *vR, *vR2;       // nR work vectors
  // PCG and direction
  double *dx, *r, *z, *p, *q, *rhs;
  double *ds, *dy, *dzl, *dzu;
  // stiff-row low-rank correction
  double* ratio;               // m
  int32_t* slotR;              // nR: slot of a stiff row, -1 otherwise
  int32_t* rowk;               // nR: constraint index of a row of R, -1 for the factor's rows
  int32_t* stiff_k;            // stiff_cap: constraint index of each slot
  int32_t* sc_cnt;             // n
  int64_t* sc_ptr;             // n+1: stiff entries per variable (CSC of the stiff rows)
  int32_t* sc_slot; double* sc_val;  // sc_cap
  int64_t sc_cap;
  double *G, *Ginv, *us, *ts;  // stiff_cap^2, stiff_cap^2, stiff_cap, stiff_cap
  double* us2;                 // stiff_cap: theta_a (A_a . p) for the exact stiff part of K~
  int stiff_cap;
  unsigned int* hist;          // kHistBins
  // dense preconditioner (n x n), nullptr if not allocated
  float2* Kd;                  // n x n pairs: the scaled condensed matrix, then its Cholesky factor (L and L^T)
  float2* Rd;                  // nR x n pairs: R as a dense matrix (when it is small enough), or nullptr
  float2* wdf;                 // nR pairs: the scaled row weights of the current dense K
  double* dense_aux;           // 4: max R^2, max |Hs| (bit patterns), the scale of K
  double* chol_diag;           // max(n_dense, stiff_cap): original diagonal during a factorisation
  double* chol_rinv;           // max(n_dense, stiff_cap): 1 / L_kk of the last factor
  double* chol_tiles;          // factored 32 x 32 diagonal tiles of the last factor (pairs for the dense K),
                               // installed into the factor by its last pass
  float2* gram_part;           // dense only, small n: partial Gram tiles of the row splits (gram_splits)
  float2* chol_rdf;            // dense only: 1 / L_kk of the dense factor (pairs)
  float2* chol_tinv;           // dense only: inverses of the dense factor's 32 x 32 diagonal tiles
  // double-float operator (storage ST_F64 with options.op_arith = DF32): the values of R and
  // R^T as (hi, lo) float32 pairs, the PCG direction p and the rows-pass result v likewise;
  // the FP64 copies stay for the residuals, the start point and the stiff-row correction
  int df;
  int mx;                      // the FP64-storage passes split their products between the float64
                               // pipe (FP64 copies) and double-float (pair copies): mixed.cu
  const float2 *R_df, *RT_df;  // nnzR each
  float2 *p_df, *v_df;         // n, nR
  // runs of R's rows: maximal stretches of consecutive entries whose columns increase by one
  // (the contiguous spot bands of a dose row), cut into pieces of at most kPiece entries; the
  // rows pass reads one descriptor per piece instead of one column index per entry when
  // `runs` is set
  int runs;
  int64_t npieces;
  const int64_t* pc_ptr;       // nR + 1: pieces of row r are [pc_ptr[r], pc_ptr[r+1])
  const int32_t* pc_col;       // npieces: column of the piece's first entry
  const uint32_t* pc_ol;       // npieces: (entry offset within the row) << 6 | length
  // tiles of the staged rows pass (staged.cu): consecutive rows [tile_row[t], tile_row[t+1])
  // whose values fit one shared-memory stage; 0 tiles = the rows pass reads global memory
  int64_t ntiles;
  const int32_t* tile_row;     // ntiles + 1
  uint64_t wait_ns;            // limit of every device-side wait (options.wait_limit_ms)
  int wait_test;               // options.wait_test: the first staged tile's wait runs out
  // gap layout of R^T for the reduced-precision column pass (lowp.cu): per column a base row
  // and 16-bit row gaps, slots padded to multiples of 8
  int gap;
  int64_t nslots;
  const int64_t* gp_ptr;       // n + 1
  const int32_t* gp_base;      // n: the column's first row
  const uint16_t* gp_d;        // nslots: row gaps
  const void* gp_q;            // nslots: narrow values (0 at fillers and padding)
  // block-Jacobi preconditioner (block.cu): blocks of 32 variables, "segments" = the entries
  // of one row of R in one block (bs_*: every row, bc_*: the constraint rows), ordered by
  // block then row; C_b (blkC, fixed per QP) and the factor of M_b (blkL), 32 x 32 each
  int64_t nblk;
  const int64_t *bs_ptr, *bs_beg, *bc_ptr, *bc_beg;   // nblk + 1 pointers; first entry of a segment
  const int32_t *bs_row, *bs_cnt, *bc_row, *bc_cnt;   // row of R and entries (<= 32) of a segment
  double *blkC, *blkL;
  // reduced-precision copy of the matrix values (storage != ST_F64): R~_ij = scaleR_i * q_ij
  int storage;
  void *Rq, *RTq;              // nnzR values each (float / bf16 / fp8-e4m3), indices shared with R, R^T
  float* scaleR;               // nR
  float *p32, *w32;            // FP32 mirror of p (n) and the rows-pass result (nR)
  double* dxr;                 // n: accumulated refined step
  double* trace;               // trace_cap rows of kTraceCols: per-IPM-iteration metrics
  // reductions and scalars
  double* partials;            // 32 * kMaxRedBlocks
  Scal* sc;
};

// (U lrs)_j by a group of G lanes over the contiguous row j of U (all lanes of the group get it).
template <int G>
__device__ __forceinline__ double lr_row(const Dev& d, const int64_t j, const bool ok, const int gl) {
  double a = 0.0;
  if (ok) {
    const double* row = d.U + j * d.ucols;
    double a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t r = gl;
    for (; r + 3 * G < d.ucols; r += 4 * G) {
      a = fma(__ldg(row + r), __ldg(d.lrs + r), a);
      a1 = fma(__ldg(row + r + G), __ldg(d.lrs + r + G), a1);
      a2 = fma(__ldg(row + r + 2 * G), __ldg(d.lrs + r + 2 * G), a2);
      a3 = fma(__ldg(row + r + 3 * G), __ldg(d.lrs + r + 3 * G), a3);
    }
    for (; r < d.ucols; r += G) a = fma(__ldg(row + r), __ldg(d.lrs + r), a);
    a = (a + a1) + (a2 + a3);
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}

constexpr int kPiece = 32;      // entries per piece of a run (at most)

// Staged rows pass (staged.cu): stages of the copy pipeline; a tile holds at most
// kStageValBytes of values, kStagePieces pieces and kStageRows rows (32 for double-float and
// 64 for the narrow storages: one row per lane group of the kStagedThreads threads).
constexpr int kStages = 3;
constexpr int kStageValBytes = 60 * 1024;
constexpr int kStagePieces = 1024;
constexpr int kStageRows = 64;
constexpr int kStageAlloc = 72 * 1024;
constexpr int kStagedThreads = 512;

// Calls f(e, c) for every stored entry e of row r of R, with its column c, by a group of G
// lanes, walking the row's pieces: the group loads G piece descriptors at a time (one per
// lane) and takes the pieces one after another, broadcast by shuffles; lane gl handles the
// piece's entries gl, gl + G, ... .  The trip counts are uniform over the warp (the most
// pieces any of its groups has; a group past its own count sees empty pieces), so every
// lane executes the same instruction stream and only masks differ.  Two pieces per trip keep
// 2 * kPiece / G entries per lane in flight; no per-entry index is read.
template <int G, typename F>
__device__ __forceinline__ void for_row_pieces(const Dev& d, const int64_t r, const bool ok, const int gl, F f) {
  const int64_t kb = ok ? d.pc_ptr[r] : 0, ke = ok ? d.pc_ptr[r + 1] : 0;
  const int64_t rb = ok ? d.R_ptr[r] : 0;
  const unsigned np = (unsigned)(ke - kb);
  const unsigned npmax = __reduce_max_sync(0xffffffffu, np);
  for (unsigned tb = 0; tb < npmax; tb += G) {
    int col = 0;
    unsigned ol = 0;
    if (tb + gl < np) {
      col = __ldg(d.pc_col + kb + tb + gl);
      ol = __ldg(d.pc_ol + kb + tb + gl);
    }
    const unsigned tn = npmax - tb < (unsigned)G ? npmax - tb : (unsigned)G;
    for (unsigned t = 0; t < tn; t += 2) {
      const int c0 = __shfl_sync(0xffffffffu, col, t, G), c1 = __shfl_sync(0xffffffffu, col, t + 1, G);
      const unsigned o0 = __shfl_sync(0xffffffffu, ol, t, G), o1 = __shfl_sync(0xffffffffu, ol, t + 1, G);
      const int len0 = (int)(o0 & 63u), len1 = t + 1 < tn ? (int)(o1 & 63u) : 0;
      const int64_t e0 = rb + (int64_t)(o0 >> 6), e1 = rb + (int64_t)(o1 >> 6);
#pragma unroll
      for (int u = 0; u < kPiece / G; ++u) {
        const int j = gl + u * G;
        if (j < len0) f(e0 + j, c0 + j);
        if (j < len1) f(e1 + j, c1 + j);
      }
    }
  }
}

// Launch geometry shared by the host code and the final reduction kernel.
struct Geo {
  int gR, gM, gN;              // blocks of the row-group kernels over R rows, constraint rows, R^T rows
  int gNc;                     // blocks of the PCG column kernels (6 resident per SM: one wave)
  int gRc;                     // blocks of the PCG row kernel (6 resident per SM: one wave)
  int gR64, gN64;              // blocks of the float64 operator passes (one wave at their occupancy)
  int gNr;                     // blocks of the residual and right-hand-side column kernels (4 per SM)
  int eM, eN;                  // blocks of the one-thread-per-element kernels over m and n
};

Geo make_geo(const Dev& d);

// Row splits of the dense Gram product: a problem with fewer 32 x 32 tiles of the lower
// triangle than about one or two per SM splits each tile's rows over 4 or 2 blocks (partial
// sums added in a fixed order), so the SMs hold more than one block each.
inline int gram_splits(int64_t n) {
  const int64_t nt = (n + 31) / 32, tiles = nt * (nt + 1) / 2;
  return tiles < 152 ? 4 : (tiles < 304 ? 2 : 1);
}

// ---- low-rank Hessian term: lrs = uw o (U^T v); quad: also v^T U W U^T v into the scalars ----
cudaError_t launch_lr(const Dev& d, const double* v, int quad, cudaStream_t st);
// ---- setup and start point ----
cudaError_t launch_diagH(const Dev& d, cudaStream_t st);
cudaError_t launch_fill_rowk(const Dev& d, cudaStream_t st);
cudaError_t launch_densify_R(const Dev& d, cudaStream_t st);   // dense.cu: Rd from R (once per QP)
cudaError_t launch_start_point(const Dev& d, const Geo& g, cudaStream_t st);
// ---- residual summary at the current iterate and mu ----
cudaError_t launch_residual_summary(const Dev& d, const Geo& g, cudaStream_t st);
// ---- complementarity residual vectors r_s, r_l, r_u (into ds, dzl, dzu) ----
cudaError_t launch_comp_resid(const Dev& d, const Geo& g, cudaStream_t st);
// ---- IPM control (mu test, stop rule, eta) ----
cudaError_t launch_control(const Dev& d, cudaStream_t st, cudaGraphConditionalHandle h = 0);
// ---- device-side IPM loop: solve start (totals reset), warm start, loop re-arming ----
cudaError_t launch_solve_begin(const Dev& d, cudaStream_t st);
cudaError_t launch_warm_start(const Dev& d, const Geo& g, cudaStream_t st);
cudaError_t launch_set_cond(cudaGraphConditionalHandle h, unsigned v, cudaStream_t st);
// ---- diagonal update and preconditioner build ----
cudaError_t launch_diag_update(const Dev& d, const Geo& g, cudaStream_t st);
cudaError_t launch_precond_build(const Dev& d, const Geo& g, int precond, cudaStream_t st);   // before rhs
cudaError_t launch_precond_finish(const Dev& d, const Geo& g, int precond, cudaStream_t st);  // after rhs
// ---- right-hand side and PCG ----
cudaError_t launch_rhs(const Dev& d, const Geo& g, int precond, cudaStream_t st);  // + Jacobi diagonal
cudaError_t launch_cg_init(const Dev& d, const Geo& g, int precond, cudaStream_t st);
cudaError_t launch_cg_body(const Dev& d, const Geo& g, int precond, cudaGraphConditionalHandle h, cudaStream_t st,
                           bool in_graph = true, bool lowp = false);
// ---- reduced-precision operator and FP64 refinement (lowp.cu) ----
cudaError_t launch_quantize(const Dev& d, cudaStream_t st);
cudaError_t launch_op_lp(const Dev& d, const Geo& g, cudaStream_t st);
cudaError_t launch_op_rows_lp_only(const Dev& d, const Geo& g, cudaStream_t st);   // measurement
cudaError_t launch_op_cols_lp_only(const Dev& d, const Geo& g, cudaStream_t st);
cudaError_t launch_mirror_p32(const Dev& d, const Geo& g, cudaStream_t st);
cudaError_t launch_gap_count(const Dev& d, int32_t* slots, cudaStream_t st);   // slots per column of R^T
cudaError_t launch_gap_fill(const Dev& d, cudaStream_t st);                    // gp_base, gp_d, gp_q
// ---- double-float operator (df.cu) ----
cudaError_t launch_df_split(const Dev& d, int* out_of_range, cudaStream_t st);   // R_df, RT_df from the FP64 values
cudaError_t launch_mirror_df(const Dev& d, const Geo& g, cudaStream_t st);        // p_df from p
cudaError_t launch_op_rows_df(const Dev& d, const Geo& g, int mode, cudaStream_t st);
cudaError_t launch_op_cols_df(const Dev& d, const Geo& g, int mode, cudaStream_t st);
// ---- split-pipe operator passes (mixed.cu) ----
cudaError_t launch_op_rows_mx(const Dev& d, const Geo& g, int mode, cudaStream_t st);
cudaError_t launch_op_cols_mx(const Dev& d, const Geo& g, int mode, cudaStream_t st);
// ---- pieces of the runs of R's rows (df.cu) ----
cudaError_t launch_runs_count(const Dev& d, int32_t* runs, int32_t* pieces, cudaStream_t st);  // per row
cudaError_t launch_runs_fill(const Dev& d, cudaStream_t st);                      // pc_col, pc_ol
cudaError_t launch_op_rows_runs(const Dev& d, const Geo& g, int mode, cudaStream_t st);   // FP64 (kernels.cu)
cudaError_t launch_op_rows_lp_runs(const Dev& d, const Geo& g, int standalone, cudaStream_t st);  // lowp.cu
// ---- staged rows pass (staged.cu): double-float or reduced storage, over pieces ----
cudaError_t launch_op_rows_staged(const Dev& d, int mode, cudaStream_t st);
cudaError_t prepare_staged();   // once per process: shared-memory limit of the staged kernels
cudaError_t launch_refine_start(const Dev& d, const Geo& g, cudaStream_t st);
// ---- reduced-precision PCG with residual replacement (lowp.cu) ----
cudaError_t launch_ru_start(const Dev& d, cudaStream_t st);
cudaError_t launch_ru_body(const Dev& d, const Geo& g, int precond, cudaGraphConditionalHandle h, cudaStream_t st,
                           bool in_graph);
cudaError_t launch_ru_end(const Dev& d, const Geo& g, cudaStream_t st);
cudaError_t launch_stiff_apply(const Dev& d, const Geo& g, cudaStream_t st);   // kernels.cu
cudaError_t launch_cg_p(const Dev& d, const Geo& g, cudaGraphConditionalHandle h, bool in_graph, cudaStream_t st);
cudaError_t launch_refine_inner(const Dev& d, const Geo& g, cudaGraphConditionalHandle hi, cudaStream_t st);
cudaError_t launch_refine_tail(const Dev& d, const Geo& g, cudaGraphConditionalHandle h, cudaStream_t st);
cudaError_t launch_refine_fallback(const Dev& d, const Geo& g, cudaStream_t st);
cudaError_t launch_refine_finish(const Dev& d, const Geo& g, cudaStream_t st);
// ---- direction recovery, ratio test, update ----
cudaError_t launch_recover(const Dev& d, const Geo& g, cudaStream_t st);
cudaError_t launch_ratio(const Dev& d, const Geo& g, cudaStream_t st);
cudaError_t launch_update(const Dev& d, const Geo& g, cudaStream_t st);
// ---- single operator apply (q = K p with the current theta, sigma) ----
cudaError_t launch_apply(const Dev& d, const Geo& g, cudaStream_t st);
// ---- the two operator kernels alone (measurement) ----
cudaError_t launch_op_rows_only(const Dev& d, const Geo& g, cudaStream_t st);
cudaError_t launch_op_cols_only(const Dev& d, const Geo& g, cudaStream_t st);
// ---- full Jacobi diagonal into Minv's storage as M (not inverted) ----
cudaError_t launch_jacobi_full(const Dev& d, const Geo& g, double* out, cudaStream_t st);

enum Precond { PC_JACOBI = 0, PC_JACOBI_LR = 1, PC_DENSE = 2, PC_BLOCK32 = 3 };
constexpr int kPrecondKinds = 4;

// ---- block-Jacobi preconditioner (block.cu) ----
cudaError_t launch_block_const(const Dev& d, cudaStream_t st);          // C_b (once per QP / cost update)
cudaError_t launch_block_factor(const Dev& d, cudaStream_t st);         // M_b and its factor (per IPM iteration)
cudaError_t launch_block_apply(const Dev& d, int init, cudaStream_t st);  // z = M^{-1} r, rz / beta

}  // namespace ipmk
