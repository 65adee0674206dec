// Solver-side entry points: implicit apply (eq. 11), projected PCG
// (Algorithm 1 with M = I) with FP64 residual replacement, recovery of alpha
// (eq. 8) and u (eq. 5), and the coarse problem set-up (eqs. 6-8).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <vector>
#include <stdexcept>
#include <string>

#include "context.h"
#include "kernels.h"

using namespace feti;

namespace {

struct CudaErr : std::runtime_error {
  using std::runtime_error::runtime_error;
};

#define CKS(x)                                                                                 \
  do {                                                                                         \
    cudaError_t e_ = (x);                                                                      \
    if (e_ != cudaSuccess) throw CudaErr(std::string(#x) + ": " + cudaGetErrorString(e_));   \
  } while (0)

// vectors inside ctx->d_vec (each n_lambda long)
// V_Q: scratch of the FP64 implicit operator; V_QK: q_k = F p_k of the iteration;
// V_Y = P M w and V_V = M w with the lumped preconditioner
enum { V_D = 0, V_R, V_W, V_P, V_Q, V_T, V_LAM0, V_LAM, V_QK, V_Y, V_V, V_U };
// coarse vectors in ctx->d_cv (each D long)
enum { C_E = 0, C_C, C_Z, C_A, C_GQ, C_C2, C_Z2 };

double* vec(feti_ctx* c, int k) { return c->d_vec + (size_t)k * c->nlam; }
double* cvec(feti_ctx* c, int k) { return c->d_cv + (size_t)k * std::max(c->dtot, 1); }

void queue_reset(feti_ctx* c, int slot) { CKS(cudaMemsetAsync(c->d_queue + slot, 0, sizeof(int), c->st)); }

// q = B L^-T L^-1 B^T p (FP64 implicit operator)
void implicit_apply(feti_ctx* c, const double* p, double* q) {
  feti_ctx::EvPair ev{};
  if (c->prof) {
    ev = {c->take_event(), c->take_event(), nullptr, nullptr, 1};
    CKS(cudaEventRecord(ev.a, c->st));
  }
  queue_reset(c, 32);
  launch_implicit(0, c->P, c->d_impl_order, c->nsub, c->d_queue + 32, p, c->d_f, c->d_qi, nullptr, c->d_uws,
                  c->ustride, c->nmax, c->impl_maxf, c->grid_impl,
                  c->impl_smem, c->st);
  launch_gather_lambda(c->d_c0, c->d_c1, c->nlam, c->d_qi, q, c->st);
  c->stats.launches += 2;
  c->stats.implicit_calls += 1;
  if (c->prof) {
    CKS(cudaEventRecord(ev.b, c->st));
    c->ev_pending.push_back(ev);
  }
}

// (G^T G)^{-1} in FP64: blocked Cholesky, inverse of the factor, W^T W
void coarse_setup(feti_ctx* c) {
  const int D = c->dtot;
  cudaStream_t st = c->st;
  if (D == 0) return;
  CKS(cudaMemsetAsync(c->d_A, 0, (size_t)D * D * 8, st));
  launch_gtg(c->d_pairs, c->npairs, c->d_plist, c->d_G6, c->d_A, D, st);
  const int nblk = (D + kT - 1) / kT;
  for (int kb = 0, b = 0; kb < D; kb += kT, ++b) {
    const int nk = std::min(kT, D - kb);
    double* Akk = c->d_A + (size_t)kb * D + kb;
    double* Dk = c->d_Dinv + (size_t)b * kT * kT;
    launch_potrf64(Akk, D, nk, Dk, c->d_status, st);
    const int rem = D - kb - nk;
    if (rem > 0) {
      double* Pan = c->d_A + (size_t)(kb + nk) * D + kb;
      launch_copy2d(Pan, D, c->d_Tp, kT, rem, nk, 1.0, st);
      // L_ik = A_ik L_kk^{-T}
      launch_gemm64(rem, nk, nk, 1.0, c->d_Tp, kT, 0, Dk, kT, 1, 0.0, Pan, D, 0, 0, st);
      // trailing lower update A_ij -= L_ik L_jk^T
      launch_gemm64(rem, rem, nk, -1.0, Pan, D, 0, Pan, D, 1, 1.0, c->d_A + (size_t)(kb + nk) * D + kb + nk, D, 1, 0,
                    st);
    }
  }
  // W = L^{-1} block row by block row: W_ii = Dinv_i, W_i,<i = -Dinv_i (L_i,<i W_<i,<i)
  CKS(cudaMemsetAsync(c->d_Linv, 0, (size_t)D * D * 8, st));
  for (int b = 0; b < nblk; ++b) {
    const int r0 = b * kT, nk = std::min(kT, D - r0);
    launch_copy2d(c->d_Dinv + (size_t)b * kT * kT, kT, c->d_Linv + (size_t)r0 * D + r0, D, nk, nk, 1.0, st);
    if (b == 0) continue;
    launch_gemm64(nk, r0, r0, 1.0, c->d_A + (size_t)r0 * D, D, 0, c->d_Linv, D, 0, 0.0, c->d_Tb, D, 0, 0, st);
    launch_gemm64(nk, r0, nk, -1.0, c->d_Dinv + (size_t)b * kT * kT, kT, 0, c->d_Tb, D, 0, 0.0,
                  c->d_Linv + (size_t)r0 * D, D, 0, 0, st);
  }
  // (G^T G)^{-1} = W^T W (K sum from max(i, j): W is lower triangular)
  launch_gemm64(D, D, D, 1.0, c->d_Linv, D, 1, c->d_Linv, D, 0, 0.0, c->d_Ainv, D, 0, 1, st);
  CKS(cudaGetLastError());
}

PcgCtrl* ctrl_dev(feti_ctx* c) { return c->d_ctrl; }
int* active_dev(feti_ctx* c) { return reinterpret_cast<int*>(reinterpret_cast<char*>(c->d_ctrl) + offsetof(PcgCtrl, active)); }

// copy the control block to pinned host memory and wait for the stream
const PcgCtrl& read_ctrl(feti_ctx* c) {
  CKS(cudaMemcpyAsync(c->h_ctrl, c->d_ctrl, sizeof(PcgCtrl), cudaMemcpyDeviceToHost, c->st));
  CKS(cudaStreamSynchronize(c->st));
  return *c->h_ctrl;
}

// y = P M w with the lumped preconditioner, the scatter of y and the dot w.y
// (mode 0: in an iteration; 1 / 2: after a residual replacement / at the start).
void enqueue_precond(feti_ctx* c, int mode, cudaStream_t st) {
  const int n = c->nlam, D = c->dtot;
  PcgCtrl* ctrl = ctrl_dev(c);
  double *w = vec(c, V_W), *y = vec(c, V_Y), *v = vec(c, V_V);
  const int iter = mode == 0 ? 1 : 0;
  if (c->precond_kind == 2) {
    // Dirichlet: v = W (sum_i B_i S_i B_i^T) W w, the M_i tiles applied by the explicit-apply tile kernel
    const auto& cand = c->apply_cands[c->apply_pick];
    launch_dir_pre(c->fp32, n, c->d_w_off, c->d_w_col, c->d_w_val, w, c->d_c0, c->d_c1, c->d_pg2, ctrl, iter, st);
    launch_apply_core(c->fp32, c->d_tdesc, c->napply, c->d_M, c->d_pg2, c->d_rowpart, c->d_tpart, cand.grid,
                      cand.variant, iter ? active_dev(c) : nullptr, c->d_status, st);
    launch_dir_mid(c->fp32, c->d_lamcol, n, c->d_rowpart, c->d_tpart, vec(c, V_U), ctrl, iter, st);
    launch_dir_post(n, c->d_w_off, c->d_w_col, c->d_w_val, vec(c, V_U), v, ctrl, iter, st);
  } else {
    launch_lumped_apply(n, c->d_w_off, c->d_w_col, c->d_w_val, c->d_m_off, c->d_m_col, c->d_m_val, w, v, ctrl,
                        iter, st);
  }
  if (D > 0) {
    launch_pcg_gt(c->P, c->nsub, c->d_G6, nullptr, v, nullptr, mode == 0 ? 2 : 3, cvec(c, C_C2), ctrl, st);
    launch_gemv_rows(c->d_Ainv, cvec(c, C_C2), cvec(c, C_Z2), D, ctrl, mode == 0 ? 2 : 1, st);
  }
  launch_pcg_proj(c->fp32, c->d_lamg, c->d_c0, c->d_c1, n, c->d_G6, D > 0 ? cvec(c, C_Z2) : nullptr, v, w, y, c->d_pg,
                  c->d_part, mode, ctrl, st);
}

// One PCPG iteration (Algorithm 1) on the device: five launches with M = I,
// nine with the lumped preconditioner; every kernel returns at once if the
// control block says the iteration has stopped.
// ev (4 events or null): before the tile kernel, around it, after the gather.
void enqueue_iteration(feti_ctx* c, double* lam, const cudaEvent_t* ev, cudaStream_t st, bool capture) {
  const unsigned evf = capture ? cudaEventRecordExternal : cudaEventRecordDefault;
  const int n = c->nlam, D = c->dtot;
  const int pre = c->precond ? 1 : 0;
  double *d = vec(c, V_D), *r = vec(c, V_R), *w = vec(c, V_W), *p = vec(c, V_P), *qk = vec(c, V_QK);
  double* y = pre ? vec(c, V_Y) : w;  // p_k = y_k + beta p_{k-1}, the apply streams F against y
  PcgCtrl* ctrl = ctrl_dev(c);
  const auto& cand = c->apply_cands[c->apply_pick];
  if (ev) CKS(cudaEventRecordWithFlags(ev[0], st, evf));
  launch_apply_core(c->fp32, c->d_tdesc, c->napply, c->d_F, c->d_pg, c->d_rowpart, c->d_tpart, cand.grid,
                    cand.variant, active_dev(c), c->d_status, st, ev ? ev[1] : nullptr, ev ? ev[2] : nullptr, capture);
  launch_pcg_gather_dot(c->fp32, c->d_lamcol, c->d_c0, c->d_c1, n, c->d_rowpart, c->d_tpart, p, y, qk, c->d_qcol,
                        c->d_part, ctrl, st);
  if (ev) CKS(cudaEventRecordWithFlags(ev[3], st, evf));
  if (D > 0) {
    launch_pcg_gt(c->P, c->nsub, c->d_G6, c->d_qcol, nullptr, nullptr, 0, cvec(c, C_GQ), ctrl, st);
    launch_gemv_rows(c->d_Ainv, cvec(c, C_GQ), cvec(c, C_Z), D, ctrl, 0, st);
  }
  launch_pcg_update(c->fp32, c->d_lamg, c->d_c0, c->d_c1, n, c->d_G6, D > 0 ? cvec(c, C_Z) : nullptr, p, qk, d, lam, r,
                    w, c->d_pg, c->d_part + kPcgMaxBlocks, 0, pre, ctrl, st);
  if (pre) enqueue_precond(c, 0, st);
}

int iteration_launches(feti_ctx* c) {
  return (c->dtot > 0 ? 5 : 3) + (c->precond ? (c->dtot > 0 ? 4 : 2) : 0) + (c->precond_kind == 2 ? 3 : 0);
}

// Capture `chunk` iterations on the private stream into one CUDA graph (once
// per context and chunk size); replaying it enqueues the whole chunk at once.
void build_chunk_graph(feti_ctx* c, double* lam, int chunk) {
  if (c->pcg_exec && c->pcg_chunk == chunk) return;
  if (c->pcg_exec) {
    CKS(cudaGraphExecDestroy(c->pcg_exec));
    c->pcg_exec = nullptr;
  }
  if (!c->cap_st) CKS(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking));
  while ((int)c->pcg_ev.size() < 4 * chunk) {
    cudaEvent_t e;
    CKS(cudaEventCreate(&e));
    c->pcg_ev.push_back(e);
  }
  cudaGraph_t g = nullptr;
  CKS(cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < chunk; ++k) enqueue_iteration(c, lam, &c->pcg_ev[4 * k], c->cap_st, true);
  cudaError_t e = cudaStreamEndCapture(c->cap_st, &g);
  if (e != cudaSuccess) throw CudaErr(std::string("capture of the PCPG chunk: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->pcg_exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) throw CudaErr(std::string("instantiation of the PCPG chunk: ") + cudaGetErrorString(e));
  c->pcg_chunk = chunk;
}

// Residual replacement with the FP64 implicit operator (eq. 11): q = F_64 lambda,
// r = d - q, w = P r (mode 1), or the start of the iteration (mode 2, which also
// sets ||w_0|| and the rounding floor).
void enqueue_refresh(feti_ctx* c, double* lam, int mode) {
  cudaStream_t st = c->st;
  const int n = c->nlam, D = c->dtot;
  double *d = vec(c, V_D), *r = vec(c, V_R), *w = vec(c, V_W), *p = vec(c, V_P), *q = vec(c, V_Q);
  PcgCtrl* ctrl = ctrl_dev(c);
  implicit_apply(c, lam, q);
  if (mode == 2) launch_pcg_norms(d, q, n, ctrl, st);
  if (D > 0) {
    launch_pcg_gt(c->P, c->nsub, c->d_G6, nullptr, q, d, 1, cvec(c, C_C), ctrl, st);
    launch_gemv_rows(c->d_Ainv, cvec(c, C_C), cvec(c, C_Z), D, ctrl, 1, st);
  }
  launch_pcg_update(c->fp32, c->d_lamg, c->d_c0, c->d_c1, n, c->d_G6, D > 0 ? cvec(c, C_Z) : nullptr, p, q, d, lam, r,
                    w, c->d_pg, c->d_part + kPcgMaxBlocks, mode, c->precond ? 1 : 0, ctrl, st);
  if (c->precond) enqueue_precond(c, mode, st);
  c->stats.launches += (D > 0 ? 3 : 1) + (mode == 2 ? 1 : 0) + (c->precond ? (D > 0 ? 4 : 2) : 0) +
                       (c->precond_kind == 2 ? 3 : 0);
}

}  // namespace

namespace feti {
// called from feti_assemble (first call): coarse problem set-up, timed as t_coarse_ms
void coarse_setup_entry(feti_ctx* c) { coarse_setup(c); }
}  // namespace feti

#define GUARD()                                                                        \
  if (!ctx) return FETI_ERR_ARG;                                                       \
  if (ctx->sticky != FETI_OK) return FETI_ERR_STATE;                                   \
  if (!ctx->assembled) return set_error(ctx, FETI_ERR_STATE, "call feti_assemble first");

extern "C" {

feti_status feti_apply_implicit(feti_ctx* ctx, const double* p_dev, double* q_dev) {
  GUARD();
  try {
    implicit_apply(ctx, p_dev, q_dev);
    CKS(cudaGetLastError());
    return FETI_OK;
  } catch (std::exception& e) {
    return set_error(ctx, FETI_ERR_CUDA, e.what());
  }
}

}  // extern "C"

namespace {

feti_status solve_impl(feti_ctx* ctx, double* lambda_dev, double* alpha_dev, double* u_dev, feti_solve_info* info,
                       bool warm) {
  GUARD();
  if (!lambda_dev) return set_error(ctx, FETI_ERR_ARG, "feti_solve: lambda_dev is required");
  try {
    cudaStream_t st = ctx->st;
    const int n = ctx->nlam;
    const int D = ctx->dtot;
    double* lam = vec(ctx, V_LAM);  // the iteration runs on an internal lambda (fixed pointers in the graph)
    double *d = vec(ctx, V_D), *r = vec(ctx, V_R), *q = vec(ctx, V_Q), *p = vec(ctx, V_P);
    // e = R^T f;  lambda_I = G (G^T G)^{-1} e
    if (D > 0) {
      launch_rtf(ctx->P, ctx->nsub, ctx->d_R, ctx->d_f, cvec(ctx, C_E), st);
      launch_gemv(ctx->d_Ainv, cvec(ctx, C_E), cvec(ctx, C_Z), D, 1.0, st);
      launch_gz(ctx->P, ctx->d_colsub, ctx->d_c0, ctx->d_c1, n, ctx->d_G6, nullptr, cvec(ctx, C_Z), -1.0, lam, st);
    } else {
      CKS(cudaMemsetAsync(lam, 0, (size_t)n * 8, st));
    }
    // d = B K^+ f - c
    queue_reset(ctx, 32);
    launch_implicit(1, ctx->P, ctx->d_impl_order, ctx->nsub, ctx->d_queue + 32, nullptr, ctx->d_f, ctx->d_qi,
                    nullptr, ctx->d_uws, ctx->ustride, ctx->nmax, ctx->impl_maxf, ctx->grid_impl, ctx->impl_smem, st);
    launch_gather_minus_c(ctx->d_c0, ctx->d_c1, n, ctx->d_qi, ctx->d_c, d, st);
    // control block; p = 0 so that the first p = w + beta p (beta = 0) is w_0
    const double tol = ctx->opt.tol > 0 ? ctx->opt.tol : 1e-10;
    const int maxit = ctx->opt.maxit > 0 ? ctx->opt.maxit : 1000;
    PcgCtrl h{};
    h.tol = tol;
    h.maxit = maxit;
    h.active = 1;
    h.restart = ctx->opt.refine_restart ? 1 : 0;
    *ctx->h_ctrl = h;
    CKS(cudaMemcpyAsync(ctx->d_ctrl, ctx->h_ctrl, sizeof(PcgCtrl), cudaMemcpyHostToDevice, st));
    // p_{-1} = q_{-1} = 0 (beta = 0 at the start, but 0 * garbage need not be 0);
    // padded B columns of pg stay 0
    CKS(cudaMemsetAsync(p, 0, (size_t)n * 8, st));
    CKS(cudaMemsetAsync(vec(ctx, V_QK), 0, (size_t)n * 8, st));
    CKS(cudaMemsetAsync(ctx->d_pg, 0, (size_t)ctx->ncols * (ctx->fp32 ? 4 : 8), st));
    // r_0 = d - F_64 lambda_I, w_0 = P r_0 (FP64 implicit operator): the reference norm and the
    // rounding floor of the stopping rule
    enqueue_refresh(ctx, lam, 2);
    if (warm) {
      // lambda_0 = lambda_g + G (G^T G)^{-1} (e - G^T lambda_g) = lambda_I + P lambda_g, then its residual
      if (D > 0) {
        launch_gt(ctx->P, ctx->nsub, ctx->d_G6, lambda_dev, cvec(ctx, C_C), st);
        launch_sub(cvec(ctx, C_E), cvec(ctx, C_C), cvec(ctx, C_C), D, st);
        launch_gemv(ctx->d_Ainv, cvec(ctx, C_C), cvec(ctx, C_Z), D, 1.0, st);
        launch_gz(ctx->P, ctx->d_colsub, ctx->d_c0, ctx->d_c1, n, ctx->d_G6, lambda_dev, cvec(ctx, C_Z), -1.0, lam,
                  st);
        ctx->stats.launches += 4;
      } else {
        CKS(cudaMemcpyAsync(lam, lambda_dev, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
      }
      enqueue_refresh(ctx, lam, 1);
    }
    PcgCtrl cur = read_ctrl(ctx);
    const double nw0 = cur.nw0;
    const int kref = ctx->opt.refine_every;
    const double drop = ctx->opt.refine_drop;
    const bool refine = kref > 0 || drop > 0.0;
    // iterations are enqueued in chunks; the host reads the control block once per chunk
    const int chunk = kref > 0 ? std::min(kref, 32) : 8;
    int nref = 0, it_ref = 0;
    double nw_ref = nw0;
    bool conv = cur.conv != 0;
    bool last_refresh = true;  // r holds d - F_64 lambda (true after the start and after a replacement)
    if (!conv) build_chunk_graph(ctx, lam, chunk);
    while (!conv && cur.it < maxit && !cur.breakdown) {
      int todo = chunk;
      if (kref > 0) todo = std::min(todo, std::max(1, kref - (cur.it - it_ref)));
      const int it0 = cur.it;
      if (todo == chunk) {
        CKS(cudaGraphLaunch(ctx->pcg_exec, st));
      } else {
        for (int k = 0; k < todo; ++k) enqueue_iteration(ctx, lam, &ctx->pcg_ev[4 * k], st, false);
      }
      ctx->stats.launches += (int64_t)todo * iteration_launches(ctx);
      cur = read_ctrl(ctx);
      const int done = cur.it - it0;  // iterations that ran (later ones returned at once)
      if (done > 0) last_refresh = false;
      ctx->stats.apply_calls += done;
      if (ctx->prof) {
        for (int k = 0; k < done; ++k) {
          float t = 0;
          CKS(cudaEventElapsedTime(&t, ctx->pcg_ev[4 * k], ctx->pcg_ev[4 * k + 3]));
          ctx->stats.apply_ms += t;
          CKS(cudaEventElapsedTime(&t, ctx->pcg_ev[4 * k + 1], ctx->pcg_ev[4 * k + 2]));
          ctx->stats.apply_tiles_ms += t;
        }
      }
      if (cur.breakdown) break;
      const bool due = refine && ((kref > 0 && cur.it - it_ref >= kref) || (drop > 0.0 && cur.nw <= drop * nw_ref) ||
                                  cur.conv);
      if (due) {
        // residual replacement (and, after the recursive residual met the stopping rule, its FP64 check)
        enqueue_refresh(ctx, lam, 1);
        cur = read_ctrl(ctx);
        last_refresh = true;
        ++nref;
        it_ref = cur.it;
        nw_ref = cur.nw;
      }
      conv = cur.conv != 0;
    }
    CKS(cudaMemcpyAsync(lambda_dev, lam, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
    // alpha = -(G^T G)^{-1} G^T (d - F lambda)  (eq. 8, FP64 implicit F).  When the iteration
    // ended on a residual replacement, r already is d - F_64 lambda for the final lambda.
    double* alpha = alpha_dev ? alpha_dev : cvec(ctx, C_A);
    if (D > 0) {
      if (!last_refresh) {
        implicit_apply(ctx, lam, q);
        launch_sub(d, q, r, n, st);
      }
      launch_gt(ctx->P, ctx->nsub, ctx->d_G6, r, cvec(ctx, C_C), st);
      launch_gemv(ctx->d_Ainv, cvec(ctx, C_C), alpha, D, -1.0, st);
    }
    // u = K^+ (f - B^T lambda) + R alpha  (eq. 5)
    if (u_dev) {
      queue_reset(ctx, 32);
      launch_implicit(2, ctx->P, ctx->d_impl_order, ctx->nsub, ctx->d_queue + 32, lam, ctx->d_f, nullptr, u_dev,
                      ctx->d_uws, ctx->ustride, ctx->nmax, ctx->impl_maxf, ctx->grid_impl, ctx->impl_smem, st);
      if (D > 0) launch_add_Ralpha(ctx->P, ctx->d_dofsub, ctx->ndof, ctx->d_R, alpha, u_dev, st);
    }
    CKS(cudaGetLastError());
    CKS(cudaStreamSynchronize(st));
    int status = 0;
    CKS(cudaMemcpy(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status & kStatTimeout) return set_error(ctx, FETI_ERR_TIMEOUT, "a bounded device wait gave up");
    if (info) {
      info->iterations = cur.it;
      info->refinements = nref;
      info->rel_residual = cur.rel;
      info->converged = conv ? 1 : 0;
      info->initial_residual = nw0;
    }
    if (!conv) return set_error(ctx, FETI_ERR_NOT_CONVERGED,
                                cur.breakdown ? "PCPG broke down (p.Fp <= 0)" : "PCPG reached maxit");
    return FETI_OK;
  } catch (std::exception& e) {
    return set_error(ctx, FETI_ERR_CUDA, e.what());
  }
}

// Z_i = P^T L_u^{-T} D^{-2} X_u (and, for the adjoint, Y_i = Z_i W_i) over batches of subdomains whose
// dense work arrays fit the budget, from X_u = L_u^{-1} P B^T recomputed in FP64 by the pruned forward
// solve with the unit-lower factor.  W_dev != null: the adjoint, dtheta_e = -sum (dK_e)_ab Y[b,:] . Z[a,:]
// into dtheta; W_dev == null: the TRSM-path assembly, F_i = B_i Z_i into the F tiles.  Synchronises.
void z_batches(feti_ctx* ctx, const double* W_dev, double* dtheta_dev, cudaStream_t st) {
  const bool adjoint = W_dev != nullptr;
  const int ns = ctx->nsub;
  if (!ctx->d_Xu) ctx->d_Xu = (double*)dalloc(ctx, (size_t)std::max<int64_t>(ctx->stats.X_elems, 1) * 8);
  queue_reset(ctx, 40);
  {
    const auto& tc = ctx->trsm_cands[ctx->trsm_pick];
    launch_trsm(ctx->P, tc.d_items, tc.nitems, tc.cw, ctx->d_queue + 40, ctx->d_Xu, false, ctx->d_ws,
                ctx->ws_stride, ctx->rhs_front, std::min(ctx->grid_trsm, tc.nitems), 0, 0, ctx->d_status, st, 1);
  }
  ctx->stats.launches += 1;
  CKS(cudaGetLastError());
  // batches of subdomains whose dense V (n x 2 m_pad, or n x m_pad for Z alone) and sorted W (m_pad^2) fit
  size_t free_b = 0, total_b = 0;
  CKS(cudaMemGetInfo(&free_b, &total_b));
  const double cap = ctx->opt.adjoint_work_bytes > 0
                         ? (double)ctx->opt.adjoint_work_bytes
                         : std::min<double>(24.0 * (1 << 30), 0.45 * (double)(free_b + ctx->adj_work_bytes));
  const int64_t budget = std::max<int64_t>((int64_t)(cap / 8), 1);
  std::vector<int64_t> woff(ns + 1, 0);
  for (int i = 0; i < ns; ++i) woff[i + 1] = woff[i] + (int64_t)ctx->subs[i].m * ctx->subs[i].m;
  std::vector<std::vector<AdjBatch>> batches;
  {
    std::vector<AdjBatch> cur;
    int64_t used = 0;
    for (int i = 0; i < ns; ++i) {
      const auto& s = ctx->subs[i];
      if (adjoint && s.nelem == 0) continue;
      if (s.m == 0) {
        if (adjoint) CKS(cudaMemsetAsync(dtheta_dev + ctx->elem_ofs[i], 0, (size_t)s.nelem * 8, st));
        continue;
      }
      const auto& I = ctx->info[i];
      const int64_t vlen = (int64_t)s.n * (adjoint ? 2 : 1) * I.m_pad;
      const int64_t need = vlen + (adjoint ? (int64_t)I.m_pad * I.m_pad : 0);
      if (!cur.empty() && used + need > budget) {
        batches.push_back(cur);
        cur.clear();
        used = 0;
      }
      AdjBatch e{};
      e.sub = i;
      e.m = s.m;
      e.m_pad = I.m_pad;
      e.zonly = adjoint ? 0 : 1;
      e.edofs = s.edofs;
      e.nelem = s.nelem;
      e.qcol = I.qcol;
      e.w_src = woff[i];
      e.v_ofs = used;
      e.ws_ofs = used + vlen;
      e.el_dofs = adjoint ? ctx->elem_dofs_ofs[i] : 0;
      e.el_dk = adjoint ? ctx->elem_dk_ofs[i] : 0;
      e.el_out = adjoint ? ctx->elem_ofs[i] : 0;
      e.dk_stride = s.dk_stride;
      cur.push_back(e);
      used += need;
    }
    if (!cur.empty()) batches.push_back(cur);
  }
  int64_t max_used = 0, max_nb = 0;
  for (auto& b : batches) {
    const AdjBatch& l = b.back();
    max_used = std::max<int64_t>(max_used, l.ws_ofs + (adjoint ? (int64_t)l.m_pad * l.m_pad : 0));
    max_nb = std::max<int64_t>(max_nb, (int64_t)b.size());
  }
  if (max_used * 8 > ctx->adj_work_bytes) {
    dfree(ctx, ctx->d_adj_work);
    ctx->d_adj_work = nullptr;
    ctx->adj_work_bytes = 0;
    ctx->d_adj_work = (double*)dalloc(ctx, (size_t)max_used * 8);
    ctx->adj_work_bytes = max_used * 8;
  }
  if (max_nb > ctx->adj_batch_cap) {
    dfree(ctx, ctx->d_adj_batch);
    ctx->d_adj_batch = (AdjBatch*)dalloc(ctx, (size_t)max_nb * sizeof(AdjBatch));
    ctx->adj_batch_cap = max_nb;
  }
  const int grid = ctx->nsm * 4;
  for (auto& b : batches) {
    const int nb = (int)b.size();
    // work items: the V rows of each (entry, active supernode, 64 own rows) and, for the adjoint, X_u W per
    // kBuildCols columns, largest first; the backward solve per (entry, 64 columns), larger factors first
    std::vector<std::pair<double, int4>> bi;
    std::vector<std::pair<double, int2>> si;
    int max_mpad = 0, max_nel = 0, max_tiles = 0;
    for (int e = 0; e < nb; ++e) {
      const auto& s = ctx->subs[b[e].sub];
      const auto& pat = ctx->pats[s.pat];
      const auto& bp = ctx->bps[s.bp];
      const int mp = b[e].m_pad;
      max_mpad = std::max(max_mpad, mp);
      max_nel = std::max(max_nel, b[e].nelem);
      max_tiles = std::max(max_tiles, bp.nb * (bp.nb + 1) / 2);
      for (int a = 0; a < (int)bp.act.size(); ++a) {
        const int sn = bp.act[a];
        const int w = pat.sn_w[sn], J = bp.je[sn] - bp.jb[sn];
        for (int k0 = 0; k0 < w; k0 += kT)
          for (int cg = 0; cg < (adjoint ? mp : 1); cg += kBuildCols)
            bi.push_back({(double)std::min(kT, w - k0) * J * (adjoint ? std::min(kBuildCols, mp - cg) : 1),
                          make_int4(e, a, k0, cg)});
      }
      for (int cb = 0; cb < (adjoint ? 2 : 1) * mp / 64; ++cb) si.push_back({pat.nnzL, make_int2(e, cb)});
    }
    std::stable_sort(bi.begin(), bi.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    std::stable_sort(si.begin(), si.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    std::vector<int4> bv;
    std::vector<int2> sv;
    bv.reserve(bi.size());
    sv.reserve(si.size());
    for (auto& x : bi) bv.push_back(x.second);
    for (auto& x : si) sv.push_back(x.second);
    if ((int64_t)bv.size() > ctx->adj_items4_cap) {
      dfree(ctx, ctx->d_adj_items4);
      ctx->d_adj_items4 = (int4*)dalloc(ctx, bv.size() * sizeof(int4));
      ctx->adj_items4_cap = (int64_t)bv.size();
    }
    if ((int64_t)sv.size() > ctx->adj_items2_cap) {
      dfree(ctx, ctx->d_adj_items2);
      ctx->d_adj_items2 = (int2*)dalloc(ctx, sv.size() * sizeof(int2));
      ctx->adj_items2_cap = (int64_t)sv.size();
    }
    // the host vectors outlive the copies: the stream is synchronised at the end of each batch
    CKS(cudaMemcpyAsync(ctx->d_adj_batch, b.data(), nb * sizeof(AdjBatch), cudaMemcpyHostToDevice, st));
    if (!bv.empty())
      CKS(cudaMemcpyAsync(ctx->d_adj_items4, bv.data(), bv.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(ctx->d_adj_items2, sv.data(), sv.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    const AdjBatch& l = b.back();
    CKS(cudaMemsetAsync(ctx->d_adj_work, 0,
                        (size_t)(l.ws_ofs + (adjoint ? (int64_t)l.m_pad * l.m_pad : 0)) * 8, st));
    if (adjoint) launch_adj_wsort(ctx->d_adj_batch, nb, W_dev, ctx->P.colperm, ctx->d_adj_work, max_mpad, st);
    queue_reset(ctx, 41);
    launch_adj_build(ctx->P, ctx->d_adj_batch, ctx->d_adj_items4, (int)bv.size(), ctx->d_queue + 41, ctx->d_Xu,
                     ctx->d_adj_work, std::max(1, std::min<int>(grid, (int)bv.size())), st);
    queue_reset(ctx, 42);
    launch_adj_bsolve(ctx->P, ctx->d_adj_batch, ctx->d_adj_items2, (int)sv.size(), ctx->d_queue + 42,
                      ctx->d_adj_work, std::max(1, std::min<int>(grid, (int)sv.size())), st);
    if (adjoint)
      launch_adj_contract(ctx->P, ctx->d_adj_batch, nb, max_nel, ctx->d_eldofs, ctx->d_eldk, ctx->d_elsc,
                          ctx->d_adj_work, dtheta_dev, st);
    else
      launch_zgather_tiles(ctx->P, ctx->d_adj_batch, nb, ctx->d_tdesc_sub, ctx->d_tile0, ctx->d_adj_work,
                           ctx->fp32, ctx->d_F, max_tiles, st);
    ctx->stats.launches += adjoint ? 4 : 3;
    CKS(cudaGetLastError());
    CKS(cudaStreamSynchronize(st));
  }
  CKS(cudaStreamSynchronize(st));
}

}  // namespace

namespace feti {
// called from feti_assemble with the TRSM-path route: F_i = B_i P^T L^{-T} X_i from the batches above
void trsm_path_entry(feti_ctx* c) { z_batches(c, nullptr, nullptr, c->st); }
}  // namespace feti

extern "C" {

feti_status feti_solve(feti_ctx* ctx, double* lambda_dev, double* alpha_dev, double* u_dev, feti_solve_info* info) {
  return solve_impl(ctx, lambda_dev, alpha_dev, u_dev, info, false);
}

feti_status feti_solve_warm(feti_ctx* ctx, double* lambda_dev, double* alpha_dev, double* u_dev,
                            feti_solve_info* info) {
  return solve_impl(ctx, lambda_dev, alpha_dev, u_dev, info, true);
}

feti_status feti_adjoint(feti_ctx* ctx, const double* W_dev, double* dtheta_dev) {
  GUARD();
  if (!W_dev || !dtheta_dev) return set_error(ctx, FETI_ERR_ARG, "feti_adjoint: W_dev and dtheta_dev are required");
  if (ctx->nelem_total == 0) return set_error(ctx, FETI_ERR_ARG, "feti_adjoint: no element data given at create");
  if (!ctx->assembled) return set_error(ctx, FETI_ERR_STATE, "feti_adjoint before feti_assemble");
  try {
    z_batches(ctx, W_dev, dtheta_dev, ctx->st);
    int status = 0;
    CKS(cudaMemcpy(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status & kStatTimeout) return set_error(ctx, FETI_ERR_TIMEOUT, "a bounded device wait gave up");
    if (ctx->opt.recompute_X) {
      // HBM is short: nothing of the adjoint is kept between calls
      dfree(ctx, ctx->d_Xu);
      ctx->d_Xu = nullptr;
      dfree(ctx, ctx->d_adj_work);
      ctx->d_adj_work = nullptr;
      ctx->adj_work_bytes = 0;
    }
    return FETI_OK;
  } catch (std::bad_alloc&) {
    return set_error(ctx, FETI_ERR_ALLOC, "feti_adjoint: device allocation failed");
  } catch (std::exception& e) {
    return set_error(ctx, FETI_ERR_CUDA, e.what());
  }
}

feti_status feti_weighted_trace(feti_ctx* ctx, const double* W_dev, double* L_dev) {
  GUARD();
  if (!W_dev || !L_dev) return set_error(ctx, FETI_ERR_ARG, "feti_weighted_trace: W_dev and L_dev are required");
  if (!ctx->assembled) return set_error(ctx, FETI_ERR_STATE, "feti_weighted_trace before feti_assemble");
  try {
    cudaStream_t st = ctx->st;
    if (!ctx->d_woff) {
      std::vector<int64_t> woff(ctx->nsub, 0);
      for (int i = 1; i < ctx->nsub; ++i) woff[i] = woff[i - 1] + (int64_t)ctx->subs[i - 1].m * ctx->subs[i - 1].m;
      ctx->d_woff = (int64_t*)dalloc(ctx, woff.size() * sizeof(int64_t));
      CKS(cudaMemcpyAsync(ctx->d_woff, woff.data(), woff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
      ctx->d_wt_part = (double*)dalloc(ctx, (size_t)std::max(ctx->napply, 1) * 8);
      CKS(cudaStreamSynchronize(st));
    }
    launch_weighted_trace(ctx->fp32, ctx->d_tdesc, ctx->napply, ctx->d_F, ctx->P.qmap, ctx->P.colsub,
                          ctx->P.colperm, ctx->P.sub, ctx->d_woff, W_dev, ctx->d_wt_part, L_dev,
                          std::max(1, std::min(ctx->napply, ctx->nsm * 8)), st);
    ctx->stats.launches += 2;
    CKS(cudaGetLastError());
    return FETI_OK;
  } catch (std::bad_alloc&) {
    return set_error(ctx, FETI_ERR_ALLOC, "feti_weighted_trace: device allocation failed");
  } catch (std::exception& e) {
    return set_error(ctx, FETI_ERR_CUDA, e.what());
  }
}

}  // extern "C"
