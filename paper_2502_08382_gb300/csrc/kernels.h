// Host-side launchers of the FETI device kernels (internal to the library).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace feti {

// flags: kCholNoReg (factor K, not K_reg), kCholStopRoot (leave the root front assembled, unfactored).
// items (subdomain, task, global task id, parent's global task id); use_tasks = 0: whole subdomains.
// tdone: per global task, child tasks finished (zeroed before the launch); hand: hand-over slots.
void launch_chol(const DevPlan& P, const int4* items, int nitems, int use_tasks, int* queue, int* tdone,
                 double* hand, double* ws, int64_t ws_stride, int64_t front_sz, int64_t stack_sz, int grid,
                 int* status, cudaStream_t st, int flags = 0);
int chol_ctas_per_sm();
// the large fronts (P.sn_big) after launch_chol with kCholSkipBig: items = the large tasks (subdomain, task,
// global task, parent's global task) children first, tdone zeroed, one CTA per SM (grid <= SMs), slices: per CTA slice_stride = chol_tc_scratch(largest front) uint16 of scratch
int64_t chol_tc_scratch(int fmax);  // uint16 elements of the per-CTA scratch for fronts up to fmax wide
void launch_chol_tc(const DevPlan& P, const int4* items, int nitems, int* queue, int* tdone, double* hand,
                    double* ws, int64_t ws_stride, int64_t front_sz, uint16_t* slices, int64_t slice_stride, int grid,
                    int* status, cudaStream_t st, int flags);
// items: (subdomain, first sorted column) pairs, each covering cw columns (cw = 0: all columns)
// X2 (FP32 X only, may be null): the bf16 hi/lo copy of X (per column: wp hi values, then wp lo values; 2 bf16
// per X element): the large fronts (P.lh_ofs >= 0, tcmode 2) use it as GEMM operand; with x2_out every
// finished block is written to it (the split-bf16 SYRK reads it)
// L32 (FP32 X only): the FP32 copy of L (launch_l32)
void launch_trsm(const DevPlan& P, const int2* items, int nitems, int cw, int* queue, void* X, bool fp32,
                 double* ws, int64_t ws_stride, int64_t front_sz, int grid, int tcmode, int tf32_out, int* status,
                 cudaStream_t st, int unit = 0, uint16_t* X2 = nullptr, const float* L32 = nullptr, int x2_out = 0);
int trsm_ctas_per_sm(bool fp32, int tcmode);
// the row-major bf16 hi/lo copies of the large panels (P.LH) and the inverses of their 32 x 32 diagonal
// blocks (P.DI) from the FP32 copy of L; items: (subdomain, local supernode) of every panel with P.lh_ofs >= 0
void launch_l16(const DevPlan& P, const int2* items, int nitems, const float* L32, uint16_t* LH, float* DI, int grid,
                cudaStream_t st);
void launch_l32(const double* L, float* L32, int64_t n, int grid, cudaStream_t st);
// X2 (split mode): the bf16 hi/lo copy of X written by the TRSM (per column: wp hi values, then wp lo values)
// variant (split mode): 0 = all threads load then one thread issues; 1 = warp-specialised (producer warps,
// issuer, epilogue warps on a double-buffered accumulator); the assembly's autotuner picks one per problem
void launch_syrk_tc(const DevPlan& P, const int2* items, int nitems, const float* X, const uint16_t* X2, float* F,
                    int grid, int split, int* status, cudaStream_t st, int variant = 0);
size_t syrk_tc_smem(int split);
void launch_syrk_f64(const DevPlan& P, const int2* items, int nitems, const double* X, double* F, int grid,
                     cudaStream_t st);
// ev_tiles0/1: optional events recorded just before / after the F-streaming kernel
void launch_apply(const DevPlan& P, bool fp32, const TileDesc* desc, int ntiles, const void* F, const int* qmap,
                  int64_t ncols, const double* p, void* pg, void* rowpart, void* colpart, const int2* blocks,
                  int nblocks, double* qi, const int* c0, const int* c1, int nlam, double* q, int grid, int variant,
                  int* status, cudaStream_t st, cudaEvent_t ev_tiles0 = nullptr, cudaEvent_t ev_tiles1 = nullptr);
void launch_apply_core(bool fp32, const TileDesc* desc, int ntiles, const void* F, const void* pg, void* rowpart,
                       void* colpart, int grid, int variant, const int* active, int* status, cudaStream_t st,
                       cudaEvent_t ev_tiles0 = nullptr, cudaEvent_t ev_tiles1 = nullptr, bool ev_external = false);
int apply_variants();
int apply_max_ctas_per_sm(bool fp32, int variant);
int apply_warps_per_cta(int variant);
void launch_unpack_F(const void* Fsub, bool fp32, int m, int nb, int vr, const int* colperm, double* out,
                     cudaStream_t st);

void launch_gather_lambda(const int* c0, const int* c1, int nlam, const double* qi, double* q, cudaStream_t st);

// FP64 solve side: implicit operator (eq. 11), K_reg solves (eqs. 5, 7),
// coarse problem and projector (eqs. 6-8), PCPG vectors (Algorithm 1)
size_t implicit_smem(int nmax, int maxf);
void launch_unit_scale(const DevPlan& P, int nsub, double* d2, cudaStream_t st);
int implicit_occupancy(size_t smem);
void launch_implicit(int mode, const DevPlan& P, const int* order, int nsub, int* queue, const double* p,
                     const double* f, double* qi, double* u, double* uws, int64_t ustride, int nmax, int maxf,
                     int grid, size_t smem, cudaStream_t st);
void launch_gather_minus_c(const int* c0, const int* c1, int nlam, const double* qi, const double* c, double* q,
                           cudaStream_t st);
void launch_build_G(const DevPlan& P, const int* colsub, int64_t ncols, const double* R, double* G6,
                    cudaStream_t st);
void launch_rtf(const DevPlan& P, int nsub, const double* R, const double* f, double* e, cudaStream_t st);
void launch_gt(const DevPlan& P, int nsub, const double* G6, const double* x, double* c, cudaStream_t st);
void launch_gz(const DevPlan& P, const int* colsub, const int* c0, const int* c1, int nlam, const double* G6,
               const double* x, const double* z, double sgn, double* out, cudaStream_t st);
void launch_gtg(const int4* pairs, int npairs, const int2* plist, const double* G6, double* A, int D,
                cudaStream_t st);
void launch_gemm64(int M, int N, int K, double alpha, const double* A, int lda, int ta, const double* B, int ldb,
                   int tb, double beta, double* C, int ldc, int lower, int ktri, cudaStream_t st);
void launch_potrf64(double* A, int lda, int n, double* Dinv, int* status, cudaStream_t st);
void launch_copy2d(const double* src, int lds, double* dst, int ldd, int rows, int cols, double scale,
                   cudaStream_t st);
// projected CG (kern_pcg.cu)
void launch_pcg_gather_dot(bool fp32, const int4* lc, const int* c0, const int* c1, int nlam, const void* rowpart,
                           const void* colpart, double* p, const double* w, double* q, double* qcol, double* part,
                           PcgCtrl* ctrl, cudaStream_t st);
void launch_pcg_gt(const DevPlan& P, int nsub, const double* G6, const double* xcol, const double* q, const double* d,
                   int mode, double* c, const PcgCtrl* ctrl, cudaStream_t st);
void launch_gemv_rows(const double* A, const double* c, double* z, int D, const PcgCtrl* ctrl, int mode,
                      cudaStream_t st);
void launch_pcg_update(bool fp32, const int4* lg, const int* c0, const int* c1, int nlam, const double* G6,
                       const double* z, const double* p, const double* q, const double* d, double* lam, double* r,
                       double* w, void* pg, double* part, int mode, int pre, PcgCtrl* ctrl, cudaStream_t st);
// lumped preconditioner (kern_pcg.cu)
void launch_lumped_values(int64_t nnz, const int64_t* c_off, const int64_t* kidx, const double* sgn,
                          const double* Kval, double* mval, cudaStream_t st);
void launch_lumped_apply(int nlam, const int* woff, const int* wcol, const double* wval, const int* moff,
                         const int* mcol, const double* mval, const double* w, double* v, const PcgCtrl* ctrl,
                         int iteration, cudaStream_t st);
// Dirichlet preconditioner (kern_pcg.cu, kern_tiles.cu)
void launch_schur_tiles(const DevPlan& P, const TileDesc* desc, int ntiles, bool fp32, void* M, int grid,
                        cudaStream_t st);
void launch_dir_pre(bool fp32, int nlam, const int* woff, const int* wcol, const double* wval, const double* w,
                    const int* c0, const int* c1, void* pg, const PcgCtrl* ctrl, int iteration, cudaStream_t st);
void launch_dir_mid(bool fp32, const int4* lc, int nlam, const void* rowpart, const void* colpart, double* u,
                    const PcgCtrl* ctrl, int iteration, cudaStream_t st);
void launch_dir_post(int nlam, const int* woff, const int* wcol, const double* wval, const double* u, double* v,
                     const PcgCtrl* ctrl, int iteration, cudaStream_t st);
void launch_pcg_proj(bool fp32, const int4* lg, const int* c0, const int* c1, int nlam, const double* G6,
                     const double* z2, const double* v, const double* w, double* y, void* pg, double* part, int mode,
                     PcgCtrl* ctrl, cudaStream_t st);
void launch_pcg_norms(const double* d, const double* q, int n, PcgCtrl* ctrl, cudaStream_t st);
void launch_sub(const double* d, const double* q, double* r, int n, cudaStream_t st);
void launch_add_Ralpha(const DevPlan& P, const int* dofsub, int64_t ndof, const double* R, const double* alpha,
                       double* u, cudaStream_t st);
void launch_gemv(const double* A, const double* c, double* z, int D, double alpha, cudaStream_t st);
// FP64 adjoint in batches of subdomains and the weighted trace (kern_adjoint.cu)
void launch_adj_wsort(const AdjBatch* B, int nb, const double* W, const int* colperm, double* work, int max_mpad,
                      cudaStream_t st);
void launch_adj_build(const DevPlan& P, const AdjBatch* B, const int4* items, int nitems, int* queue,
                      const double* Xu, double* work, int grid, cudaStream_t st);
void launch_adj_bsolve(const DevPlan& P, const AdjBatch* B, const int2* items, int nitems, int* queue, double* work,
                       int grid, cudaStream_t st);
void launch_adj_contract(const DevPlan& P, const AdjBatch* B, int nb, int max_nelem, const int* eldofs,
                         const double* eldk, const double* elsc, const double* work, double* g, cudaStream_t st);
// TRSM-path assembly: F_i tiles from the rows of Z_i = K_reg^{-1} B_i^T at the B DOFs (desc: tiles in
// subdomain-major order, tile0: the subdomain's first tile)
void launch_zgather_tiles(const DevPlan& P, const AdjBatch* B, int nb, const TileDesc* desc, const int* tile0,
                          const double* work, bool fp32, void* F, int max_tiles, cudaStream_t st);
void launch_weighted_trace(bool fp32, const TileDesc* desc, int ntiles, const void* F, const int* qmap,
                           const int* colsub, const int* colperm, const SubInfo* sub, const int64_t* woff,
                           const double* W, double* part, double* out, int grid, cudaStream_t st);
}  // namespace feti
