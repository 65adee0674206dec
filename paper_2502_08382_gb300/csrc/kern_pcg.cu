// Vector kernels of the projected conjugate gradient (Algorithm 1, M = I),
// fused so that one iteration is five launches and no host round trip:
//
//   1. tiles:    the F-streaming tile kernel (kern_apply.cu) on pg = B w_k,
//                gathered into the tile precision by the previous update;
//   2. gather:   f = F w_k from the tile partials (Algorithm 2's gather); by
//                linearity of F, q_k = F p_k = f + beta q_{k-1} and
//                p_k = w_k + beta p_{k-1}; the dot p.q, whose last block sets
//                delta = (w.w) / (p.q); q_k is also written per B column;
//   3. G^T q_k per subdomain, from the per-column copy;
//   4. z -= delta (G^T G)^{-1} G^T q_k  (explicit FP64 inverse, eqs. 6-8): z
//                follows r, z_k = (G^T G)^{-1} G^T r_k;
//   5. update:   lambda += delta p, r -= delta q (or r = d - F lambda on a
//                residual replacement), w = r - G z (the projector), the dot
//                w.w and the scatter pg = B w for the next iteration; the last
//                block sets beta, the relative residual and the stop flags.
//
// The control block lives in device memory; every kernel of an iteration
// returns at once when `active` is 0, so the host can enqueue several
// iterations ahead and read the control block once per chunk.  Dot products
// are reduced in a fixed order (block partials summed by one block), so a
// solve is bitwise reproducible.  Per-multiplier index data is precomputed on
// the host so that every thread starts its loads from one coalesced record.
#include "common.cuh"
#include "kernels.h"

namespace feti {
namespace {

constexpr int kVT = 256;  // threads per block of the vector kernels

// Sum a double over the block in a fixed order; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)blockDim.x / 32; ++k) s += red[k];
  __syncthreads();
  return s;
}

// Store the block partial; returns true (in every thread) for the last block
// to arrive, after which all partials are visible to it.
__device__ __forceinline__ bool last_block(double s, double* part, int* counter) {
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    __threadfence();
    is_last = atomicAdd(counter, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last != 0;
}

// Fixed-order sum of the nb block partials by one block (thread 0 holds it).
__device__ __forceinline__ double sum_partials(const double* part, int nb, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  return block_sum(s, red);
}

// One thread per multiplier l.  lc[l] = {tile base, (column << 8) | nb} of
// its first and second subdomain column (second tile base -1 if none): f =
// colsum(first) + colsum(second), both in the fixed order of colsum_at.
template <typename TF>
__global__ void __launch_bounds__(kVT) pcg_gather_dot_kernel(const int4* lc, const int* c0, const int* c1, int nlam,
                                                             const TF* rowpart, const TF* colpart, double* p,
                                                             const double* w, double* q, double* qcol, double* part,
                                                             PcgCtrl* ctrl) {
  __shared__ double red[kVT / 32];
  if (!ctrl->active) return;
  const double beta = ctrl->beta;
  double s = 0.0;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlam; l += gridDim.x * blockDim.x) {
    const int4 c = lc[l];
    double f = colsum_at((int64_t)c.x, c.y & 255, c.y >> 8, rowpart, colpart);
    if (c.z >= 0) f += colsum_at((int64_t)c.z, c.w & 255, c.w >> 8, rowpart, colpart);
    const double ql = fma(beta, q[l], f);
    const double pl = fma(beta, p[l], w[l]);
    q[l] = ql;
    p[l] = pl;
    qcol[c0[l]] = ql;
    const int b = c1[l];
    if (b >= 0) qcol[b] = ql;
    s = fma(pl, ql, s);
  }
  s = block_sum(s, red);
  if (last_block(s, part, &ctrl->cnt_dot)) {
    const double pq = sum_partials(part, gridDim.x, red);
    if (threadIdx.x == 0) {
      ctrl->pq = pq;
      if (pq > 0.0 && isfinite(pq)) {
        ctrl->delta = ctrl->wy / pq;
      } else {  // breakdown: F p is not positive on p (Algorithm 1 needs F SPD on ker G^T)
        ctrl->delta = 0.0;
        ctrl->breakdown = 1;
        ctrl->active = 0;
      }
      ctrl->cnt_dot = 0;
    }
  }
}

// c[alpha0 + k] = sum_j G[(qcol + j), k] x_j with x = the per-column copy of
// q (mode 0, iteration), (d - q)[map_j] (mode 1, residual replacement) or
// q[map_j] (mode 2 in an iteration, mode 3 in a replacement; the
// preconditioned vector); modes 0 and 2 return at once when the iteration has
// stopped.  One warp per (subdomain, k), loads four columns ahead.
__global__ void pcg_gt_kernel(DevPlan P, int nsub, const double* G6, const double* xcol, const double* q,
                              const double* d, int mode, double* c, const PcgCtrl* ctrl) {
  if ((mode == 0 || mode == 2) && !ctrl->active) return;
  const int lane = threadIdx.x & 31;
  for (int wk = (blockIdx.x * blockDim.x + threadIdx.x) / 32; wk < nsub * 6; wk += gridDim.x * blockDim.x / 32) {
    const int si = wk / 6, k = wk % 6;
    const SubInfo& S = P.sub[si];
    if (k >= S.d) continue;
    double acc = 0.0;
#pragma unroll 4
    for (int j = lane; j < S.m; j += 32) {
      const int64_t g = S.qcol + j;
      double x;
      if (mode == 0) {
        x = xcol[g];
      } else {
        const int l = P.qmap[g];
        x = mode == 1 ? d[l] - q[l] : q[l];
      }
      acc = fma(G6[g * 6 + k], x, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) c[S.alpha0 + k] = acc;
  }
}

// mode 1: z = A c;  mode 0 (iteration): z -= delta A c;  mode 2: z = A c in an
// iteration.  Modes 0 and 2 return at once when the iteration has stopped.  A
// dense D x D row-major; 4 rows per block, 2 warps per row, fixed-order sums
__global__ void __launch_bounds__(kVT) gemv_rows_kernel(const double* A, const double* c, double* z, int D,
                                                        const PcgCtrl* ctrl, int mode) {
  __shared__ double red[kVT / 32];
  if (ctrl && mode != 1 && !ctrl->active) return;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 4 + warp / 2, half = warp & 1;
  double acc = 0.0;
  if (row < D) {
    const double* a = A + (int64_t)row * D;
    for (int j = half * 32 + lane; j < D; j += 64) acc = fma(a[j], c[j], acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x < 4 && blockIdx.x * 4 + threadIdx.x < D) {
    const int64_t i = blockIdx.x * 4 + threadIdx.x;
    const double v = red[2 * threadIdx.x] + red[2 * threadIdx.x + 1];
    z[i] = mode == 0 ? fma(-ctrl->delta, v, z[i]) : v;
  }
}

// beta and w.y after the dot wyn = w.y of the new iterate: mode 0 (iteration)
// beta = wyn / (w.y before), mode 2 (start) beta = 0, mode 1 (residual
// replacement) the replaced residual takes the place of this iteration's
// recursive one: beta divides by the w.y the iteration started from, or the
// search direction restarts (iterative refinement with inner CG solves).
__device__ __forceinline__ void set_direction(PcgCtrl* ctrl, double wyn, int mode) {
  ctrl->wyn = wyn;
  if (mode == 2) {
    ctrl->beta = 0.0;
    ctrl->wy_prev = wyn;
  } else if (mode == 0) {
    ctrl->beta = ctrl->wy > 0.0 ? wyn / ctrl->wy : 0.0;
    ctrl->wy_prev = ctrl->wy;
  } else {
    ctrl->beta = ctrl->restart ? 0.0 : (ctrl->wy_prev > 0.0 ? wyn / ctrl->wy_prev : 0.0);
  }
  ctrl->wy = wyn;
}

// mode 0 (iteration): lambda += delta p, r -= delta q;  mode 1 (refresh): r = d - q;  mode 2 (start): as 1,
// and the start values nw0 / floor are set.  Then w = r - G z, the dot w.w and the scatter of w into the
// tile precision for the next apply (pg at both B columns of the multiplier); the last block finishes.
// lg[l] = {alpha0, d} of the first and the second subdomain of l (d = 0 if none).
template <typename TF>
__global__ void __launch_bounds__(kVT) pcg_update_kernel(const int4* lg, const int* c0, const int* c1, int nlam,
                                                         const double* G6, const double* z, const double* p,
                                                         const double* q, const double* d, double* lam, double* r,
                                                         double* w, TF* pg, double* part, int mode, int pre,
                                                         PcgCtrl* ctrl) {
  __shared__ double red[kVT / 32];
  if (mode == 0 && !ctrl->active) return;
  const double delta = ctrl->delta;
  double s = 0.0;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlam; l += gridDim.x * blockDim.x) {
    double rl;
    if (mode == 0) {
      lam[l] = fma(delta, p[l], lam[l]);
      rl = fma(-delta, q[l], r[l]);
    } else {
      rl = d[l] - q[l];
    }
    r[l] = rl;
    const int g0 = c0[l], g1 = c1[l];
    double gz = 0.0;
    if (z) {
      const int4 a = lg[l];
      for (int k = 0; k < a.y; ++k) gz = fma(G6[(int64_t)g0 * 6 + k], z[a.x + k], gz);
      for (int k = 0; k < a.w; ++k) gz = fma(G6[(int64_t)g1 * 6 + k], z[a.z + k], gz);
    }
    const double wl = rl - gz;
    w[l] = wl;
    if (!pre) {  // with a preconditioner the apply streams F against y = P M w, scattered later
      pg[g0] = (TF)wl;
      if (g1 >= 0) pg[g1] = (TF)wl;
    }
    s = fma(wl, wl, s);
  }
  s = block_sum(s, red);
  if (last_block(s, part, &ctrl->cnt_upd)) {
    const double wyn = sum_partials(part, gridDim.x, red);
    if (threadIdx.x == 0) {
      const double nw = sqrt(wyn);  // wyn = w.w here
      ctrl->nw = nw;
      if (mode == 2) {
        // start: floor = 64 eps (||d|| + ||F lambda_0||) from the two norms stored before
        ctrl->nw0 = nw;
        ctrl->floor = 64.0 * 2.220446049250313e-16 * (sqrt(ctrl->dd) + sqrt(ctrl->qq));
      }
      if (!pre) set_direction(ctrl, wyn, mode);  // M = I: y = w
      if (mode == 0) ctrl->it += 1;
      ctrl->rel = ctrl->nw0 > 0.0 ? nw / ctrl->nw0 : 0.0;
      ctrl->conv = (nw <= ctrl->tol * ctrl->nw0 || nw <= ctrl->floor) ? 1 : 0;
      ctrl->active = (!ctrl->conv && !ctrl->breakdown && ctrl->it < ctrl->maxit) ? 1 : 0;
      ctrl->cnt_upd = 0;
    }
  }
}

// ---------------------------------------------------------------- lumped preconditioner
//
// M = W M_core W with W = (B B^T)^{-1} (small dense blocks, CSR) and
// M_core = sum_i B_i K_i B_i^T (CSR over multipliers; its values are summed
// from K at every assembly).  y = P M w needs v = M w, its projection and the
// dot w.y; the apply of the next iteration then streams F against y.

// mval[e] = sum of the entry's (sign, K value) contributions, in stored order
__global__ void lumped_values_kernel(int64_t nnz, const int64_t* c_off, const int64_t* kidx, const double* sgn,
                                     const double* Kval, double* mval) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int64_t k = c_off[e]; k < c_off[e + 1]; ++k) v = fma(sgn[k], Kval[kidx[k]], v);
    mval[e] = v;
  }
}

// v = W M_core W w, one thread per multiplier a:
//   v_a = sum_{c in W row a} W_ac sum_{e in M_core row c} m_e sum_{f in W row col_e} W_{col_e f} w_f
// (W's blocks are a node's few multipliers, so the redundant inner sums are short).
__global__ void __launch_bounds__(kVT) lumped_apply_kernel(int nlam, const int* woff, const int* wcol,
                                                           const double* wval, const int* moff, const int* mcol,
                                                           const double* mval, const double* w, double* v,
                                                           const PcgCtrl* ctrl, int iteration) {
  if (iteration && !ctrl->active) return;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nlam; a += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = woff[a]; i < woff[a + 1]; ++i) {
      const int c = wcol[i];
      double sc = 0.0;
      for (int e = moff[c]; e < moff[c + 1]; ++e) {
        const int d = mcol[e];
        double t = 0.0;
        for (int f = woff[d]; f < woff[d + 1]; ++f) t = fma(wval[f], w[wcol[f]], t);
        sc = fma(mval[e], t, sc);
      }
      acc = fma(wval[i], sc, acc);
    }
    v[a] = acc;
  }
}

// Dirichlet preconditioner v = W (sum_i B_i S_i B_i^T) W w in three vector steps around the tile apply of the
// M_i = B_i S_i B_i^T tiles: t = W w scattered to both subdomain columns of each multiplier in the tile
// precision (dir_pre), the tiles (apply core), u = the two column sums per multiplier (dir_mid), v = W u
// (dir_post).  In an iteration (iteration = 1) every kernel returns at once once the iteration has stopped.
template <typename TF>
__global__ void __launch_bounds__(kVT) dir_pre_kernel(int nlam, const int* woff, const int* wcol, const double* wval,
                                                      const double* w, const int* c0, const int* c1, TF* pg,
                                                      const PcgCtrl* ctrl, int iteration) {
  if (iteration && !ctrl->active) return;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlam; l += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int i = woff[l]; i < woff[l + 1]; ++i) t = fma(wval[i], w[wcol[i]], t);
    pg[c0[l]] = (TF)t;
    if (c1[l] >= 0) pg[c1[l]] = (TF)t;
  }
}

template <typename TF>
__global__ void __launch_bounds__(kVT) dir_mid_kernel(const int4* lc, int nlam, const TF* rowpart, const TF* colpart,
                                                      double* u, const PcgCtrl* ctrl, int iteration) {
  if (iteration && !ctrl->active) return;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlam; l += gridDim.x * blockDim.x) {
    const int4 c = lc[l];
    double f = colsum_at((int64_t)c.x, c.y & 255, c.y >> 8, rowpart, colpart);
    if (c.z >= 0) f += colsum_at((int64_t)c.z, c.w & 255, c.w >> 8, rowpart, colpart);
    u[l] = f;
  }
}

__global__ void __launch_bounds__(kVT) dir_post_kernel(int nlam, const int* woff, const int* wcol, const double* wval,
                                                       const double* u, double* v, const PcgCtrl* ctrl,
                                                       int iteration) {
  if (iteration && !ctrl->active) return;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlam; l += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int i = woff[l]; i < woff[l + 1]; ++i) t = fma(wval[i], u[wcol[i]], t);
    v[l] = t;
  }
}

// y = v - G z2 (the projection of v = M w; z2 = (G^T G)^{-1} G^T v, or none
// without a coarse space), the scatter of y into the tile precision for the
// next apply, and the dot w.y; the last block sets beta and w.y (set_direction).
// mode 0 (iteration) returns at once when the iteration has stopped.
template <typename TF>
__global__ void __launch_bounds__(kVT) pcg_proj_kernel(const int4* lg, const int* c0, const int* c1, int nlam,
                                                       const double* G6, const double* z2, const double* v,
                                                       const double* w, double* y, TF* pg, double* part, int mode,
                                                       PcgCtrl* ctrl) {
  __shared__ double red[kVT / 32];
  if (mode == 0 && !ctrl->active) return;
  double s = 0.0;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlam; l += gridDim.x * blockDim.x) {
    const int g0 = c0[l], g1 = c1[l];
    double gz = 0.0;
    if (z2) {
      const int4 a = lg[l];
      for (int k = 0; k < a.y; ++k) gz = fma(G6[(int64_t)g0 * 6 + k], z2[a.x + k], gz);
      for (int k = 0; k < a.w; ++k) gz = fma(G6[(int64_t)g1 * 6 + k], z2[a.z + k], gz);
    }
    const double yl = v[l] - gz;
    y[l] = yl;
    pg[g0] = (TF)yl;
    if (g1 >= 0) pg[g1] = (TF)yl;
    s = fma(w[l], yl, s);
  }
  s = block_sum(s, red);
  if (last_block(s, part, &ctrl->cnt_proj)) {
    const double wyn = sum_partials(part, gridDim.x, red);
    if (threadIdx.x == 0) {
      set_direction(ctrl, wyn, mode);
      ctrl->cnt_proj = 0;
    }
  }
}

// dd = d.d and qq = q.q (for the rounding floor of the stopping rule), one block
__global__ void __launch_bounds__(kVT) pcg_norms_kernel(const double* d, const double* q, int n, PcgCtrl* ctrl) {
  __shared__ double red[kVT / 32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a = fma(d[i], d[i], a);
    b = fma(q[i], q[i], b);
  }
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    ctrl->dd = a;
    ctrl->qq = b;
  }
}

inline int vgrid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + kVT - 1) / kVT, kPcgMaxBlocks)); }

}  // namespace

void launch_pcg_gather_dot(bool fp32, const int4* lc, const int* c0, const int* c1, int nlam, const void* rowpart,
                           const void* colpart, double* p, const double* w, double* q, double* qcol, double* part,
                           PcgCtrl* ctrl, cudaStream_t st) {
  if (fp32)
    pcg_gather_dot_kernel<float><<<vgrid(nlam), kVT, 0, st>>>(lc, c0, c1, nlam, (const float*)rowpart,
                                                             (const float*)colpart, p, w, q, qcol, part, ctrl);
  else
    pcg_gather_dot_kernel<double><<<vgrid(nlam), kVT, 0, st>>>(lc, c0, c1, nlam, (const double*)rowpart,
                                                              (const double*)colpart, p, w, q, qcol, part, ctrl);
}

void launch_pcg_gt(const DevPlan& P, int nsub, const double* G6, const double* xcol, const double* q, const double* d,
                   int mode, double* c, const PcgCtrl* ctrl, cudaStream_t st) {
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)nsub * 6 * 32 + kVT - 1) / kVT, 152 * 16));
  pcg_gt_kernel<<<g, kVT, 0, st>>>(P, nsub, G6, xcol, q, d, mode, c, ctrl);
}

void launch_gemv_rows(const double* A, const double* c, double* z, int D, const PcgCtrl* ctrl, int mode,
                      cudaStream_t st) {
  if (D > 0) gemv_rows_kernel<<<(D + 3) / 4, kVT, 0, st>>>(A, c, z, D, ctrl, mode);
}

void launch_pcg_update(bool fp32, const int4* lg, const int* c0, const int* c1, int nlam, const double* G6,
                       const double* z, const double* p, const double* q, const double* d, double* lam, double* r,
                       double* w, void* pg, double* part, int mode, int pre, PcgCtrl* ctrl, cudaStream_t st) {
  if (fp32)
    pcg_update_kernel<float><<<vgrid(nlam), kVT, 0, st>>>(lg, c0, c1, nlam, G6, z, p, q, d, lam, r, w, (float*)pg,
                                                          part, mode, pre, ctrl);
  else
    pcg_update_kernel<double><<<vgrid(nlam), kVT, 0, st>>>(lg, c0, c1, nlam, G6, z, p, q, d, lam, r, w, (double*)pg,
                                                           part, mode, pre, ctrl);
}

void launch_lumped_values(int64_t nnz, const int64_t* c_off, const int64_t* kidx, const double* sgn,
                          const double* Kval, double* mval, cudaStream_t st) {
  if (nnz <= 0) return;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((nnz + kVT - 1) / kVT, 152 * 16));
  lumped_values_kernel<<<g, kVT, 0, st>>>(nnz, c_off, kidx, sgn, Kval, mval);
}

void launch_lumped_apply(int nlam, const int* woff, const int* wcol, const double* wval, const int* moff,
                         const int* mcol, const double* mval, const double* w, double* v, const PcgCtrl* ctrl,
                         int iteration, cudaStream_t st) {
  lumped_apply_kernel<<<vgrid(nlam), kVT, 0, st>>>(nlam, woff, wcol, wval, moff, mcol, mval, w, v, ctrl, iteration);
}

void launch_dir_pre(bool fp32, int nlam, const int* woff, const int* wcol, const double* wval, const double* w,
                    const int* c0, const int* c1, void* pg, const PcgCtrl* ctrl, int iteration, cudaStream_t st) {
  if (fp32)
    dir_pre_kernel<float><<<vgrid(nlam), kVT, 0, st>>>(nlam, woff, wcol, wval, w, c0, c1, (float*)pg, ctrl, iteration);
  else
    dir_pre_kernel<double><<<vgrid(nlam), kVT, 0, st>>>(nlam, woff, wcol, wval, w, c0, c1, (double*)pg, ctrl,
                                                        iteration);
}

void launch_dir_mid(bool fp32, const int4* lc, int nlam, const void* rowpart, const void* colpart, double* u,
                    const PcgCtrl* ctrl, int iteration, cudaStream_t st) {
  if (fp32)
    dir_mid_kernel<float><<<vgrid(nlam), kVT, 0, st>>>(lc, nlam, (const float*)rowpart, (const float*)colpart, u,
                                                       ctrl, iteration);
  else
    dir_mid_kernel<double><<<vgrid(nlam), kVT, 0, st>>>(lc, nlam, (const double*)rowpart, (const double*)colpart, u,
                                                        ctrl, iteration);
}

void launch_dir_post(int nlam, const int* woff, const int* wcol, const double* wval, const double* u, double* v,
                     const PcgCtrl* ctrl, int iteration, cudaStream_t st) {
  dir_post_kernel<<<vgrid(nlam), kVT, 0, st>>>(nlam, woff, wcol, wval, u, v, ctrl, iteration);
}

void launch_pcg_proj(bool fp32, const int4* lg, const int* c0, const int* c1, int nlam, const double* G6,
                     const double* z2, const double* v, const double* w, double* y, void* pg, double* part, int mode,
                     PcgCtrl* ctrl, cudaStream_t st) {
  if (fp32)
    pcg_proj_kernel<float><<<vgrid(nlam), kVT, 0, st>>>(lg, c0, c1, nlam, G6, z2, v, w, y, (float*)pg, part, mode,
                                                        ctrl);
  else
    pcg_proj_kernel<double><<<vgrid(nlam), kVT, 0, st>>>(lg, c0, c1, nlam, G6, z2, v, w, y, (double*)pg, part, mode,
                                                         ctrl);
}

void launch_pcg_norms(const double* d, const double* q, int n, PcgCtrl* ctrl, cudaStream_t st) {
  pcg_norms_kernel<<<1, kVT, 0, st>>>(d, q, n, ctrl);
}

}  // namespace feti
