// Internal definition of feti_ctx (host runtime state).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "feti.h"
#include "common.cuh"
#include "symbolic.h"

namespace feti {

struct SubHost {
  int n = 0, m = 0, d = 0, nfix = 0, nelem = 0, edofs = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  std::vector<int32_t> bdof, blam;
  std::vector<double> bsign;
  std::vector<double> R, f, coords;
  std::vector<int32_t> fix;
  std::vector<int32_t> elem_dofs;
  std::vector<double> dKe, dKe_scale;  // per element (dk_stride = edofs^2) or one shared matrix (0)
  int64_t dk_stride = 0;
  int pat = -1, bp = -1;
};

// a device buffer owned by the context
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace feti

struct feti_ctx {
  feti_options opt{};
  cudaStream_t st = nullptr;
  std::string err;
  feti_status sticky = FETI_OK;
  int nsub = 0, nlam = 0, nsm = 0;
  bool fp32 = false;
  bool assembled = false;
  std::vector<double> c_host;
  std::vector<feti::SubHost> subs;
  std::vector<feti::PatternPlan> pats;
  std::vector<feti::BPlan> bps;
  std::vector<int> bp_pat;
  std::vector<feti::SubInfo> info;
  feti::DevPlan P{};
  std::vector<feti::DBuf> bufs;
  size_t device_bytes = 0;
  // device arrays not in DevPlan
  double* d_Kval = nullptr;
  double* d_L = nullptr;
  void* d_X = nullptr;
  void* d_F = nullptr;
  double* d_ws = nullptr;
  int64_t ws_stride = 0, chol_front = 0, rhs_front = 0, chol_stack = 0;
  double* d_trow = nullptr;
  double* d_tpart = nullptr;
  double* d_qi = nullptr;
  int* d_colsub = nullptr;
  int* d_c0 = nullptr;
  int* d_c1 = nullptr;
  int* d_queue = nullptr;     // [8] work-queue counters
  int* d_status = nullptr;    // [1]
  int* d_chol_order = nullptr;
  int* d_trsm_order = nullptr;
  struct TrsmCand {
    int cw;           // columns per work item (0: a whole subdomain)
    int2* d_items;    // (subdomain, first column), subdomains by decreasing TRSM cost
    int nitems;
    double ms;
  };
  std::vector<TrsmCand> trsm_cands;  // autotuner candidates of the pruned TRSM
  int trsm_pick = 0;
  bool trsm_tuned = false;
  int4* d_chol_items[2] = {nullptr, nullptr};  // Cholesky items: whole subdomains / subtree tasks
  int chol_nitems[2] = {0, 0};
  int chol_pick = 0;                 // the autotuner's choice of the two
  bool chol_tuned = false;
  int ntask_total = 0;
  int* d_tdone = nullptr;            // per global task: child tasks finished
  double* d_hand = nullptr;          // hand-over slots of split subtree roots
  int4* d_tc_items = nullptr;        // the large fronts' tasks (the tensor-core Cholesky's items)
  int n_tc_items = 0, grid_tc = 0;
  uint16_t* d_slices = nullptr;      // its per-CTA scratch (bf16 slices and row exponents)
  int64_t slice_stride = 0;
  int2* d_l16_items = nullptr;       // (subdomain, supernode) of the panels with a row-major hi/lo copy
  int n_l16 = 0;
  int syrk_variant = 0;              // split-bf16 SYRK kernel picked by the autotuner
  bool syrk_tuned = false;
  int* d_impl_order = nullptr;
  int2* d_syrk_items = nullptr;
  feti::TileDesc* d_tdesc = nullptr;
  struct ApplyCand {
    int variant, grid;  // tile-kernel variant (load batch) and grid
    double ms;
  };
  std::vector<ApplyCand> apply_cands;  // autotuner candidates of the apply
  int apply_pick = 0;
  bool apply_tuned = false;
  void* d_pg = nullptr;
  void* d_rowpart = nullptr;
  int2* d_syrk2_items = nullptr;
  int2* d_blocks = nullptr;
  int nblocks = 0;
  int nsyrk2 = 0;
  int* d_colperm = nullptr;   // per subdomain sorted column -> B row (for get_F)
  std::vector<int64_t> colperm_ofs;
  int nsyrk = 0, napply = 0;
  int64_t ncols = 0;
  int grid_chol = 0, grid_trsm = 0, grid_impl = 0;
  int grid_trsm32 = 0;  // CTAs of the mixed-precision TRSM (its occupancy with the tensor-core stage ring)
  size_t impl_smem = 0;
  double* d_uws = nullptr;  // update vectors of the implicit solve, ustride doubles per CTA
  int64_t ustride = 0;
  int impl_maxf = 0;
  // solve-side data
  bool coarse_ready = false;
  int npairs = 0;
  int4* d_pairs = nullptr;
  int2* d_plist = nullptr;
  double* d_G6 = nullptr;      // [ncols * 6] G = B R per sorted column
  double* d_A = nullptr;       // D x D coarse matrix, then its factor
  double* d_Ainv = nullptr;    // (G^T G)^{-1}
  double* d_Linv = nullptr;
  double* d_Dinv = nullptr;    // inverses of the 64 x 64 diagonal factor blocks
  double* d_Tp = nullptr;      // D x 64 panel scratch
  double* d_Tb = nullptr;      // 64 x D row-block scratch
  int4* d_lamcol = nullptr;    // per multiplier: tile bases and columns of its subdomain columns (PCPG gather)
  int4* d_lamg = nullptr;      // per multiplier: alpha0 and d of its subdomains (PCPG update)
  double* d_qcol = nullptr;    // per B column: q of its multiplier (PCPG G^T q)
  int m_max = 0;               // widest subdomain (B rows)
  // lumped preconditioner M = W M_core W (options.precond = 1), see precond.cpp
  bool precond = false;
  int precond_kind = 0;        // 0 none, 1 lumped, 2 Dirichlet
  feti::DevPlan P2{};          // Dirichlet: the plan with its own L (K factored up to the root front) and rho
  void* d_M = nullptr;         // Dirichlet: M_i = B_i S_i B_i^T tiles (layout of F)
  void* d_pg2 = nullptr;       // Dirichlet: W w gathered per sorted column (tile precision)
  int* d_w_off = nullptr;
  int* d_w_col = nullptr;
  double* d_w_val = nullptr;
  int* d_m_off = nullptr;
  int* d_m_col = nullptr;
  double* d_m_val = nullptr;
  int64_t* d_mc_off = nullptr;
  int64_t* d_mc_kidx = nullptr;
  double* d_mc_sign = nullptr;
  int64_t m_nnz = 0;
  double* d_vec = nullptr;     // PCPG vectors (11 x n_lambda)
  double* d_cv = nullptr;      // coarse vectors (7 x D)
  double* d_sc = nullptr;      // scalars
  double* d_part = nullptr;    // block partials of the PCPG reductions (2 x kPcgMaxBlocks)
  double* h_sc = nullptr;      // pinned host scalars
  feti::PcgCtrl* d_ctrl = nullptr;  // PCPG control block
  feti::PcgCtrl* h_ctrl = nullptr;  // pinned host copy
  cudaStream_t cap_st = nullptr;     // private stream on which CUDA graphs are captured
  cudaGraphExec_t asm_exec = nullptr;  // the numeric assembly (Cholesky, TRSM, scaling, SYRK), replayed on st
  void* asm_X = nullptr;             // the X buffers the assembly graph was captured with
  void* asm_X2 = nullptr;
  uint16_t* d_X2 = nullptr;          // bf16 hi/lo copy of X (split-bf16 SYRK operands)
  float* d_L32 = nullptr;            // FP32 copy of L for the mixed TRSM
  cudaGraphExec_t pcg_exec = nullptr;  // captured chunk of iterations (replayed on st)
  int pcg_chunk = 0;
  std::vector<cudaEvent_t> pcg_ev;  // 4 events per captured iteration (apply timing)
  int* d_dofsub = nullptr;
  // adjoint (element data and dense work buffers, allocated on first use)
  std::vector<int64_t> elem_ofs, elem_dk_ofs, elem_dofs_ofs;
  int* d_ident = nullptr;
  int64_t nelem_total = 0;
  int* d_eldofs = nullptr;
  double* d_eldk = nullptr;
  double* d_elsc = nullptr;
  double* d_Xu = nullptr;          // FP64 X_u = L_u^{-1} P B^T of every subdomain (adjoint)
  double* d_adj_work = nullptr;    // batch work arrays of the adjoint (V and sorted W)
  int64_t adj_work_bytes = 0;
  feti::AdjBatch* d_adj_batch = nullptr;
  int64_t adj_batch_cap = 0;
  int4* d_adj_items4 = nullptr;
  int64_t adj_items4_cap = 0;
  int2* d_adj_items2 = nullptr;
  feti::TileDesc* d_tdesc_sub = nullptr;  // the apply's tile descriptors in subdomain-major order
  int* d_tile0 = nullptr;                 // first tile of each subdomain in d_tdesc_sub
  int route = 0;                          // assembly route in use (0 SYRK path, 1 Schur, 2 TRSM path)
  bool route_tuned = false;
  double route_ms[3] = {0, 0, 0};
  int64_t adj_items2_cap = 0;
  int64_t* d_woff = nullptr;       // per subdomain offset of W_i (weighted trace)
  double* d_wt_part = nullptr;     // per tile partials of the weighted trace
  int64_t ndof = 0;
  int nmax = 0;
  double* d_R = nullptr;       // concatenated R_i (column-major n x d)
  double* d_f = nullptr;       // concatenated f_i
  double* d_c = nullptr;       // c
  int dtot = 0;
  // stats and measurement
  feti_stats stats{};
  bool prof = false;
  struct EvPair {
    cudaEvent_t a, b, c, d;
    int kind;  // 0 apply (a..d whole, b..c tiles), 1 implicit (a..b)
  };
  std::vector<EvPair> ev_pending;
  std::vector<cudaEvent_t> ev_pool;
  cudaEvent_t take_event() {
    if (ev_pool.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      return e;
    }
    cudaEvent_t e = ev_pool.back();
    ev_pool.pop_back();
    return e;
  }
  cudaEvent_t ev[8]{};
};

namespace feti {
feti_status set_error(feti_ctx* c, feti_status s, const std::string& msg);
void trsm_path_entry(feti_ctx* c);  // the TRSM-path assembly of the F_i tiles (api_solve.cpp)
void* dalloc(feti_ctx* c, size_t bytes);
void dfree(feti_ctx* c, void* p);  // release a buffer from dalloc (no-op for nullptr)
}  // namespace feti
