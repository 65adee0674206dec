// Solver-side entry points: implicit apply (eq. 11), projected PCG
// (Algorithm 1 with M = I) with FP64 residual replacement, recovery of alpha
// (eq. 8) and u (eq. 5), and the coarse problem set-up (eqs. 6-8).
#include <cmath>
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

constexpr int kNPart = 512;

// vectors inside ctx->d_vec (each n_lambda long)
enum { V_D = 0, V_R, V_W, V_P, V_Q, V_T, V_LAM0 };
// scalars in ctx->d_sc
enum { S_WY = 0, S_PQ = 1, S_WYN = 2, S_TMP = 3 };
// coarse vectors in ctx->d_cv (each D long)
enum { C_E = 0, C_C, C_Z, C_A };

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

// out = P x = x - G (G^T G)^{-1} G^T x
void project(feti_ctx* c, const double* x, double* out) {
  if (c->dtot == 0) {
    if (out != x) CKS(cudaMemcpyAsync(out, x, (size_t)c->nlam * 8, cudaMemcpyDeviceToDevice, c->st));
    return;
  }
  launch_gt(c->P, c->nsub, c->d_G6, x, cvec(c, C_C), c->st);
  launch_gemv(c->d_Ainv, cvec(c, C_C), cvec(c, C_Z), c->dtot, 1.0, c->st);
  launch_gz(c->P, c->d_colsub, c->d_c0, c->d_c1, c->nlam, c->d_G6, x, cvec(c, C_Z), 1.0, out, c->st);
  c->stats.launches += 3;
}

double dot_host(feti_ctx* c, const double* x, const double* y, int slot) {
  launch_dot(x, y, c->nlam, c->d_part, kNPart, c->d_sc + slot, c->st);
  c->stats.launches += 2;
  CKS(cudaMemcpyAsync(c->h_sc + slot, c->d_sc + slot, 8, cudaMemcpyDeviceToHost, c->st));
  CKS(cudaStreamSynchronize(c->st));
  return c->h_sc[slot];
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

feti_status feti_solve(feti_ctx* ctx, double* lambda_dev, double* alpha_dev, double* u_dev, feti_solve_info* info) {
  GUARD();
  if (!lambda_dev) return set_error(ctx, FETI_ERR_ARG, "feti_solve: lambda_dev is required");
  try {
    cudaStream_t st = ctx->st;
    const int n = ctx->nlam;
    const int D = ctx->dtot;
    double* lam = lambda_dev;
    double *d = vec(ctx, V_D), *r = vec(ctx, V_R), *w = vec(ctx, V_W), *p = vec(ctx, V_P), *q = vec(ctx, V_Q);
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
    // r0 = d - F lambda_0 (FP64 implicit), w0 = P r0, y0 = w0 (M = I), p0 = y0
    implicit_apply(ctx, lam, q);
    launch_sub(d, q, r, n, st);
    project(ctx, r, w);
    CKS(cudaMemcpyAsync(p, w, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
    double wy = dot_host(ctx, w, w, S_WY);
    const double nw0 = std::sqrt(wy);
    const double tol = ctx->opt.tol > 0 ? ctx->opt.tol : 1e-10;
    const int maxit = ctx->opt.maxit > 0 ? ctx->opt.maxit : 1000;
    const int kref = ctx->opt.refine_every;
    int it = 0, nref = 0;
    bool conv = nw0 == 0.0;
    double rel = nw0 == 0.0 ? 0.0 : 1.0;
    while (!conv && it < maxit) {
      // q = F p (explicit, stored precision); delta = (w.y) / (p.q)
      feti_status s = feti_apply(ctx, p, q);
      if (s != FETI_OK) return s;
      launch_dot(p, q, n, ctx->d_part, kNPart, ctx->d_sc + S_PQ, st);
      launch_pcg_upd1(lam, r, p, q, ctx->d_sc, n, st);
      ctx->stats.launches += 3;
      ++it;
      bool refined = false;
      if (kref > 0 && it % kref == 0) {
        // residual replacement with the FP64 implicit operator
        implicit_apply(ctx, lam, q);
        launch_sub(d, q, r, n, st);
        ctx->stats.launches += 1;
        ++nref;
        refined = true;
      }
      project(ctx, r, w);
      double wyn = dot_host(ctx, w, w, S_WYN);
      rel = std::sqrt(wyn) / nw0;
      if (rel <= tol) {
        if (kref > 0 && !refined) {
          implicit_apply(ctx, lam, q);
          launch_sub(d, q, r, n, st);
          ++nref;
          project(ctx, r, w);
          wyn = dot_host(ctx, w, w, S_WYN);
          rel = std::sqrt(wyn) / nw0;
        }
        if (rel <= tol) {
          conv = true;
          break;
        }
      }
      // p = y + beta p, beta = (w_new . y_new) / (w . y)
      launch_pcg_upd2(p, w, ctx->d_sc, n, st);
      launch_scalar_copy(ctx->d_sc, S_WY, S_WYN, st);
      ctx->stats.launches += 2;
      wy = wyn;
    }
    // alpha = -(G^T G)^{-1} G^T (d - F lambda)  (eq. 8, FP64 implicit F)
    double* alpha = alpha_dev ? alpha_dev : cvec(ctx, C_A);
    if (D > 0) {
      implicit_apply(ctx, lam, q);
      launch_sub(d, q, r, n, st);
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
      info->iterations = it;
      info->refinements = nref;
      info->rel_residual = rel;
      info->converged = conv ? 1 : 0;
    }
    if (!conv) return set_error(ctx, FETI_ERR_NOT_CONVERGED, "PCPG reached maxit");
    return FETI_OK;
  } catch (std::exception& e) {
    return set_error(ctx, FETI_ERR_CUDA, e.what());
  }
}

feti_status feti_adjoint(feti_ctx* ctx, const double* W_dev, double* dtheta_dev) {
  GUARD();
  if (!W_dev || !dtheta_dev) return set_error(ctx, FETI_ERR_ARG, "feti_adjoint: W_dev and dtheta_dev are required");
  if (ctx->nelem_total == 0) return set_error(ctx, FETI_ERR_ARG, "feti_adjoint: no element data given at create");
  try {
    cudaStream_t st = ctx->st;
    size_t zmax = 0;
    for (auto& s : ctx->subs)
      if (s.nelem > 0) zmax = std::max(zmax, (size_t)s.n * s.m);
    if (!ctx->d_Z) {
      ctx->d_Z = (double*)dalloc(ctx, std::max<size_t>(zmax, 1) * 8);
      ctx->d_Y = (double*)dalloc(ctx, std::max<size_t>(zmax, 1) * 8);
    }
    int64_t woff = 0;
    for (int i = 0; i < ctx->nsub; ++i) {
      const auto& s = ctx->subs[i];
      const int n = s.n, m = s.m;
      if (s.nelem > 0 && m > 0) {
        // Z = K_reg^{-1} B^T (rows: original DOFs, columns: B rows), FP64, recomputed here
        queue_reset(ctx, 33);
        launch_implicit(3, ctx->P, ctx->d_ident + i, m, ctx->d_queue + 33, nullptr, nullptr, nullptr, ctx->d_Z,
                        ctx->d_uws, ctx->ustride, ctx->nmax, ctx->impl_maxf, ctx->grid_impl, ctx->impl_smem, st);
        // Y = Z W_i
        launch_gemm64(n, m, m, 1.0, ctx->d_Z, m, 0, W_dev + woff, m, 0, 0.0, ctx->d_Y, m, 0, 0, st);
        // dtheta_e = -scale_e <dK_ref, (Y Z^T)_e>
        launch_elem_contract(ctx->d_eldofs + ctx->elem_dofs_ofs[i], s.nelem, s.edofs, ctx->d_eldk + ctx->elem_dk_ofs[i],
                             ctx->d_elsc + ctx->elem_ofs[i], ctx->d_Z, ctx->d_Y, m, dtheta_dev + ctx->elem_ofs[i], st);
        ctx->stats.launches += 3;
      } else if (s.nelem > 0) {
        CKS(cudaMemsetAsync(dtheta_dev + ctx->elem_ofs[i], 0, (size_t)s.nelem * 8, st));
      }
      woff += (int64_t)m * m;
    }
    CKS(cudaGetLastError());
    CKS(cudaStreamSynchronize(st));
    return FETI_OK;
  } catch (std::exception& e) {
    return set_error(ctx, FETI_ERR_CUDA, e.what());
  }
}

}  // extern "C"
