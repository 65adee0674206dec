// FP64 solve-side kernels:
//  * implicit operator (paper eq. 11) and the solves with K_reg used by d
//    (eq. 7) and the primal recovery (eq. 5): supernodal forward / backward
//    substitution with L_i, one subdomain per CTA, the subdomain vector held
//    in shared memory;
//  * the coarse problem G^T G (G = B R, eqs. 6-8): deterministic assembly,
//    blocked Cholesky and explicit inverse built from 64 x 64 FP64 tile GEMMs;
//  * the projector P = I - G (G^T G)^{-1} G^T and the PCPG vector updates of
//    Algorithm 1 (M = I), with dot products reduced in a fixed order.
#include "common.cuh"
#include "kernels.h"

namespace feti {
namespace {

constexpr int kW = 32;

__device__ __forceinline__ int pop_item_s(int* queue) {
  __shared__ int item;
  __syncthreads();
  if (threadIdx.x == 0) item = atomicAdd(queue, 1);
  __syncthreads();
  return item;
}

constexpr int kWF = 128;  // largest front handled by one warp (needs w <= 32)

// The implicit solves use L in unit-lower form, L = Lu D (D = diag of L),
// written by unit_scale_kernel after the assembly: the panel holds Lu below
// the diagonal and zeros on and above it, and d2[j] = 1 / L_jj^2.  Then
// K_reg^{-1} y = Lu^{-T} D^{-2} Lu^{-1} y: the forward sweep needs no pivot
// and its own entries are scaled by d2 once, the backward sweep none.

// One warp: forward step of a small supernode (w <= 32, w + r <= kWF).  Lane
// l keeps the front entries l + 32 q in registers; per column j, z_j comes
// from lane j and every front row takes its update in one FMA (the zeros of
// Lu on and above the diagonal leave the rows <= j unchanged).
__device__ __forceinline__ void fwd_warp(const DevPlan& P, const SubInfo& S, int gs, const double* d2,
                                         double* ubuf, double* y, double* v, int lane) {
  const int c0 = P.sn_c0[gs], w = P.sn_w[gs], r = P.sn_r[gs], f_ = w + r;
  const double* Ls = P.L + S.L + P.Lofs[gs];
  for (int i = lane; i < f_; i += 32) v[i] = i < w ? y[c0 + i] : 0.0;
  __syncwarp();
  for (int c = P.ch_off[gs]; c < P.ch_off[gs + 1]; ++c) {
    const int gc = S.sn0 + P.ch_list[c];
    const int rc = P.sn_r[gc];
    const double* U = ubuf + P.uofs[gc];
    const int* rl = P.rel + P.rel_off[gc];
    for (int k = lane; k < rc; k += 32) v[rl[k]] += U[k];
    __syncwarp();
  }
  const int nq = (f_ + 31) / 32;  // warp-uniform
  double a[kWF / 32];
#pragma unroll
  for (int q = 0; q < kWF / 32; ++q) {
    const int i = lane + 32 * q;
    a[q] = (q < nq && i < f_) ? v[i] : 0.0;
  }
  // columns in groups of 4: the group's loads are issued together, so one
  // global-memory latency is paid per group instead of per column
  constexpr int kU = 4;
  for (int j0 = 0; j0 < w; j0 += kU) {
    double lc[kU][kWF / 32];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int j = j0 + u;
      const double* col = Ls + (int64_t)j * f_;
#pragma unroll
      for (int q = 0; q < kWF / 32; ++q) {
        const int i = lane + 32 * q;
        lc[u][q] = (j < w && q < nq && i < f_) ? col[i] : 0.0;
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int j = j0 + u;
      if (j >= w) break;
      const double zj = __shfl_sync(0xffffffffu, a[0], j);
#pragma unroll
      for (int q = 0; q < kWF / 32; ++q)
        if (q < nq) a[q] = fma(-lc[u][q], zj, a[q]);
    }
  }
  if (lane < w) y[c0 + lane] = a[0] * d2[c0 + lane];
  double* Us = ubuf + P.uofs[gs];
#pragma unroll
  for (int q = 0; q < kWF / 32; ++q) {
    const int i = lane + 32 * q;
    if (i >= w && i < f_) Us[i - w] = a[q];
  }
  __syncwarp();
}

// One warp: backward step of a small supernode.  The rows part
// t_l = sum_i L21[i][l] x_rows[i] is split over G = 32 / 2^ceil(log2 w)
// row groups per column (lane = l + wp g), reduced with shuffles; then lane
// l owns x_l through the triangular sweep.
__device__ __forceinline__ void bwd_warp(const DevPlan& P, const SubInfo& S, int gs, double* y, double* v,
                                         int lane) {
  const int c0 = P.sn_c0[gs], w = P.sn_w[gs], r = P.sn_r[gs], f_ = w + r;
  const double* Ls = P.L + S.L + P.Lofs[gs];
  const int* rows = P.rows + P.sn_rows[gs];
  for (int i = lane; i < r; i += 32) v[i] = y[rows[i]];
  __syncwarp();
  int wp = 1;
  while (wp < w) wp <<= 1;
  const int G = 32 / wp, l = lane % wp, g = lane / wp;
  double t = 0.0;
  if (l < w) {
    const double* col = Ls + (int64_t)l * f_ + w;
#pragma unroll 4
    for (int i = g; i < r; i += G) t = fma(col[i], v[i], t);
  }
  for (int o = wp; o < 32; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  double x = lane < w ? y[c0 + lane] - t : 0.0;
  for (int j0 = w - 1; j0 >= 0; j0 -= 4) {
    double lr[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = j0 - u;
      lr[u] = (j >= 0 && lane < j) ? Ls[(int64_t)lane * f_ + j] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = j0 - u;
      if (j < 0) break;
      const double xj = __shfl_sync(0xffffffffu, x, j);
      x = fma(-lr[u], xj, x);
    }
  }
  if (lane < w) y[c0 + lane] = x;
  __syncwarp();
}

// Whole CTA: forward step of a large supernode on the shared front vector.
// 32 x 32 unit-lower diagonal blocks are staged in shared memory and solved
// by warp 0; all threads apply the block's columns to the rest of the front.
__device__ __forceinline__ void fwd_cta(const DevPlan& P, const SubInfo& S, int gs, const double* d2,
                                        double* ubuf, double* y, double* sf, double (*sm_blk)[kW + 1], int tid) {
  const int warp = tid / 32, lane = tid % 32;
  const int c0 = P.sn_c0[gs], w = P.sn_w[gs], r = P.sn_r[gs], f_ = w + r;
  const double* Ls = P.L + S.L + P.Lofs[gs];
  for (int i = tid; i < f_; i += kThreads) sf[i] = i < w ? y[c0 + i] : 0.0;
  __syncthreads();
  for (int c = P.ch_off[gs]; c < P.ch_off[gs + 1]; ++c) {
    const int gc = S.sn0 + P.ch_list[c];
    const int rc = P.sn_r[gc];
    const double* U = ubuf + P.uofs[gc];
    const int* rl = P.rel + P.rel_off[gc];
    for (int k = tid; k < rc; k += kThreads) sf[rl[k]] += U[k];
    __syncthreads();
  }
  for (int kb = 0; kb < w; kb += kW) {
    const int nbk = min(kW, w - kb);
    for (int idx = tid; idx < nbk * kW; idx += kThreads) {
      const int k = idx / kW, i = idx % kW;  // column k, row i of the block
      if (i < nbk) sm_blk[i][k] = (i >= k) ? Ls[(int64_t)(kb + k) * f_ + kb + i] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      double yi = lane < nbk ? sf[kb + lane] : 0.0;
      for (int k = 0; k < nbk; ++k) {
        const double yk = __shfl_sync(0xffffffffu, yi, k);
        yi = fma(-sm_blk[lane][k], yk, yi);  // zero on and above the diagonal
      }
      if (lane < nbk) sf[kb + lane] = yi;
    }
    __syncthreads();
    // rows in pairs (i, i + kThreads) per thread, so that each group of column loads has twice the bytes in
    // flight; a last unpaired row alone.  Every row's sum runs over k in the same order either way.
    int i = kb + nbk + tid;
    for (; i + kThreads < f_; i += 2 * kThreads) {
      double acc = 0.0, acc2 = 0.0;
#pragma unroll 8
      for (int k = 0; k < nbk; ++k) {
        const double* col = Ls + (int64_t)(kb + k) * f_;
        const double zk = sf[kb + k];
        acc = fma(col[i], zk, acc);
        acc2 = fma(col[i + kThreads], zk, acc2);
      }
      sf[i] -= acc;
      sf[i + kThreads] -= acc2;
    }
    if (i < f_) {
      double acc = 0.0;
#pragma unroll 8
      for (int k = 0; k < nbk; ++k) acc = fma(Ls[(int64_t)(kb + k) * f_ + i], sf[kb + k], acc);
      sf[i] -= acc;
    }
    __syncthreads();
  }
  double* Us = ubuf + P.uofs[gs];
  for (int i = tid; i < f_; i += kThreads) {
    if (i < w) y[c0 + i] = sf[i] * d2[c0 + i];
    else Us[i - w] = sf[i];
  }
  __syncthreads();
}

// Whole CTA: backward step of a large supernode (x_rows already final).  The
// entries x_rows are gathered into sf first; then each warp takes kBC own
// columns at a time, so their column loads are in flight together (the dot
// product of each column runs over the rows in the same order as with one
// column per warp, and is reduced the same way).
constexpr int kBC = 4;
__device__ __forceinline__ void bwd_cta(const DevPlan& P, const SubInfo& S, int gs, double* y, double* sf,
                                        double (*sm_blk)[kW + 1], int tid) {
  const int warp = tid / 32, lane = tid % 32;
  const int c0 = P.sn_c0[gs], w = P.sn_w[gs], r = P.sn_r[gs], f_ = w + r;
  const double* Ls = P.L + S.L + P.Lofs[gs];
  const int* rows = P.rows + P.sn_rows[gs];
  for (int k = tid; k < r; k += kThreads) sf[k] = y[rows[k]];
  __syncthreads();
  for (int l0 = warp * kBC; l0 < w; l0 += (kThreads / 32) * kBC) {
    if (l0 + kBC <= w) {
      double acc[kBC];
      const double* col[kBC];
#pragma unroll
      for (int u = 0; u < kBC; ++u) {
        acc[u] = 0.0;
        col[u] = Ls + (int64_t)(l0 + u) * f_ + w;
      }
#pragma unroll 2
      for (int k = lane; k < r; k += 32) {
        const double xk = sf[k];
#pragma unroll
        for (int u = 0; u < kBC; ++u) acc[u] = fma(col[u][k], xk, acc[u]);
      }
#pragma unroll
      for (int u = 0; u < kBC; ++u) {
        double a = acc[u];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) y[c0 + l0 + u] -= a;
      }
    } else {
      // the last w mod kBC columns one at a time (warp-uniform branch)
      for (int l = l0; l < w; ++l) {
        const double* col = Ls + (int64_t)l * f_ + w;
        double a = 0.0;
#pragma unroll 4
        for (int k = lane; k < r; k += 32) a = fma(col[k], sf[k], a);
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) y[c0 + l] -= a;
      }
    }
  }
  __syncthreads();
  for (int kb = ((w - 1) / kW) * kW; kb >= 0; kb -= kW) {
    const int nbk = min(kW, w - kb);
    if (nbk == kW) {
      // a full block: the warp's columns l = kb + warp + 8 u all at once
      constexpr int kU = kW / (kThreads / 32);
      double acc[kU];
      const double* col[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        acc[u] = 0.0;
        col[u] = Ls + (int64_t)(kb + warp + (kThreads / 32) * u) * f_;
      }
#pragma unroll 2
      for (int i = kb + nbk + lane; i < w; i += 32) {
        const double xi = y[c0 + i];
#pragma unroll
        for (int u = 0; u < kU; ++u) acc[u] = fma(col[u][i], xi, acc[u]);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        double a = acc[u];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) y[c0 + kb + warp + (kThreads / 32) * u] -= a;
      }
    } else {
      for (int l = kb + warp; l < kb + nbk; l += kThreads / 32) {
        double acc = 0.0;
#pragma unroll 4
        for (int i = kb + nbk + lane; i < w; i += 32) acc = fma(Ls[(int64_t)l * f_ + i], y[c0 + i], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) y[c0 + l] -= acc;
      }
    }
    for (int idx = tid; idx < nbk * kW; idx += kThreads) {
      const int k = idx / kW, i = idx % kW;
      if (i < nbk) sm_blk[i][k] = (i >= k) ? Ls[(int64_t)(kb + k) * f_ + kb + i] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      double yi = lane < nbk ? y[c0 + kb + lane] : 0.0;
      for (int k = nbk - 1; k >= 0; --k) {
        const double yk = __shfl_sync(0xffffffffu, yi, k);
        yi = fma(-sm_blk[k][lane], yk, yi);  // zero on and above the diagonal
      }
      if (lane < nbk) y[c0 + kb + lane] = yi;
    }
    __syncthreads();
  }
}

// MODE 0: qi = B L^-T L^-1 P B^T p        (implicit apply, eq. 11)
// MODE 1: qi = B K_reg^{-1} f             (d = B K^+ f - c, eq. 7)
// MODE 2: u  = K_reg^{-1} (f - B^T lambda) (eq. 5 without R alpha)
// MODE 3: column j of Z = K_reg^{-1} B^T for one subdomain (items = its
//         sorted columns; `nsub` is the column count, order[0] the subdomain);
//         written to u as Z[dof * m + B-row of column j] (original DOF order)
template <int MODE>
__global__ void __launch_bounds__(kThreads, 4) implicit_kernel(DevPlan P, const int* order, int nsub, int* queue,
                                                             const double* p, const double* f, double* qi,
                                                             double* u, double* uws, int64_t ustride, int nmax,
                                                             int maxf) {
  extern __shared__ double y[];  // [nmax] subdomain vector, [maxf] front, [8 kWF] warp fronts
  __shared__ double sm_blk[kW][kW + 1];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  double* sfront = y + nmax;
  double* wbuf = sfront + maxf;
  double* ubuf = uws + (int64_t)blockIdx.x * ustride;
  for (;;) {
    const int itx = pop_item_s(queue);
    if (itx >= nsub) return;
    const int si = MODE == 3 ? order[0] : order[itx];
    const SubInfo& S = P.sub[si];
    const int n = S.n;
    const double* d2 = P.dinv + S.dof;  // 1 / L_jj^2 (unit-lower form)
    for (int k = tid; k < n; k += kThreads) y[k] = 0.0;
    __syncthreads();
    if (MODE == 3 && tid == 0) y[P.spos[S.col0 + itx]] = P.qsign[S.qcol + itx];
    if (MODE == 1 || MODE == 2)
      for (int k = tid; k < n; k += kThreads) y[P.iperm[S.diag0 + k]] = f[S.dof + k];
    __syncthreads();
    if (MODE == 0 || MODE == 2) {
      // B^T p: columns sharing a DOF are adjacent in sorted order; the first of a run sums it
      const int* sp = P.spos + S.col0;
      for (int j = tid; j < S.m; j += kThreads) {
        if (j > 0 && sp[j - 1] == sp[j]) continue;
        double s = 0.0;
        for (int jj = j; jj < S.m && sp[jj] == sp[j]; ++jj) s += P.qsign[S.qcol + jj] * p[P.qmap[S.qcol + jj]];
        y[sp[j]] += (MODE == 0) ? s : -s;
      }
    }
    __syncthreads();
    // forward substitution L z = y, level by level from the leaves of the
    // supernodal tree.  Supernodes of one level are independent: each one
    // assembles its front vector from its own columns of y and the update
    // vectors of its children (in fixed order, so the result is
    // deterministic), solves with its diagonal block and writes its own
    // update vector for the parent.  Small fronts take one warp each, large
    // ones the whole CTA.
    const int* lvo = P.lvl_off + S.lvl0;
    const int* lsn = P.lvl_sn;
    for (int l = 0; l < S.nlev; ++l) {
      const int lo = lvo[l], hi = lvo[l + 1];
      for (int it = lo + warp; it < hi; it += kThreads / 32) {
        const int gs = S.sn0 + lsn[it];
        const int w = P.sn_w[gs], f_ = w + P.sn_r[gs];
        if (w > 32 || f_ > kWF) continue;
        fwd_warp(P, S, gs, d2, ubuf, y, wbuf + warp * kWF, lane);
      }
      __syncthreads();
      for (int it = lo; it < hi; ++it) {
        const int gs = S.sn0 + lsn[it];
        const int w = P.sn_w[gs], f_ = w + P.sn_r[gs];
        if (w <= 32 && f_ <= kWF) continue;
        fwd_cta(P, S, gs, d2, ubuf, y, sfront, sm_blk, tid);
      }
    }
    // backward substitution L^T x = z, level by level from the roots; every
    // supernode reads only ancestors' entries of x and writes its own columns
    for (int l = S.nlev - 1; l >= 0; --l) {
      const int lo = lvo[l], hi = lvo[l + 1];
      for (int it = lo + warp; it < hi; it += kThreads / 32) {
        const int gs = S.sn0 + lsn[it];
        const int w = P.sn_w[gs], f_ = w + P.sn_r[gs];
        if (w > 32 || f_ > kWF) continue;
        bwd_warp(P, S, gs, y, wbuf + warp * kWF, lane);
      }
      __syncthreads();
      for (int it = lo; it < hi; ++it) {
        const int gs = S.sn0 + lsn[it];
        const int w = P.sn_w[gs], f_ = w + P.sn_r[gs];
        if (w <= 32 && f_ <= kWF) continue;
        bwd_cta(P, S, gs, y, sfront, sm_blk, tid);
      }
    }
    __syncthreads();
    if (MODE == 0 || MODE == 1) {
      for (int j = tid; j < S.m_pad; j += kThreads)
        qi[S.qcol + j] = j < S.m ? P.qsign[S.qcol + j] * y[P.spos[S.col0 + j]] : 0.0;
    } else if (MODE == 2) {
      for (int k = tid; k < n; k += kThreads) u[S.dof + k] = y[P.iperm[S.diag0 + k]];
    } else {
      const int col = P.colperm[S.qcol + itx];  // B row of this sorted column
      for (int k = tid; k < n; k += kThreads) u[(int64_t)k * S.m + col] = y[P.iperm[S.diag0 + k]];
    }
    __syncthreads();
  }
}

// Unit-lower form of every factor, for the implicit solves (after the TRSM,
// which uses L itself): column j of each panel is divided by L_jj, the
// diagonal is set to zero and d2[dof + j] = 1 / L_jj^2.  One CTA per
// subdomain: the pivots' reciprocals are gathered first (into d2), then every
// panel is scaled with coalesced accesses, then d2 is squared.
__global__ void __launch_bounds__(256) unit_scale_kernel(DevPlan P, int nsub, double* d2) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int si = blockIdx.x; si < nsub; si += gridDim.x) {
    const SubInfo& S = P.sub[si];
    double* inv = d2 + S.dof;
    for (int s = warp; s < S.nsn; s += 8) {
      const int gs = S.sn0 + s;
      const int c0 = P.sn_c0[gs], w = P.sn_w[gs], f_ = w + P.sn_r[gs];
      const double* Ls = P.L + S.L + P.Lofs[gs];
      for (int k = lane; k < w; k += 32) inv[c0 + k] = 1.0 / Ls[(int64_t)k * f_ + k];
    }
    __syncthreads();
    for (int s = warp; s < S.nsn; s += 8) {
      const int gs = S.sn0 + s;
      const int c0 = P.sn_c0[gs], w = P.sn_w[gs], f_ = w + P.sn_r[gs];
      double* Ls = P.L + S.L + P.Lofs[gs];
      const int ne = f_ * w;
      for (int e = lane; e < ne; e += 32) {
        const int k = e / f_, i = e - k * f_;
        if (i > k) Ls[e] *= inv[c0 + k];
        else if (i == k) Ls[e] = 0.0;
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < S.n; j += blockDim.x) inv[j] *= inv[j];
    __syncthreads();
  }
}

// q[l] = qi[c0] + qi[c1] - c[l]
__global__ void gather_minus_c_kernel(const int* c0, const int* c1, int nlam, const double* qi, const double* c,
                                      double* q) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlam; l += gridDim.x * blockDim.x) {
    const int a = c0[l], b = c1[l];
    double s = a >= 0 ? qi[a] : 0.0;
    if (b >= 0) s += qi[b];
    q[l] = s - (c ? c[l] : 0.0);
  }
}

// ---------------------------------------------------------------- G = B R

// G6[g * 6 + k] = sign_j R_i[dof_j, k] for sorted column g of subdomain i
__global__ void build_G_kernel(DevPlan P, const int* colsub, int64_t ncols, const double* R, double* G6) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ncols; g += (int64_t)gridDim.x * blockDim.x) {
    const SubInfo& S = P.sub[colsub[g]];
    const int j = (int)(g - S.qcol);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      double v = 0.0;
      if (j < S.m && k < S.d) v = P.qsign[g] * R[S.R + (int64_t)k * S.n + P.qdof[g]];
      G6[g * 6 + k] = v;
    }
  }
}

// e[alpha0 + k] = R_i[:, k]^T f_i ; one warp per (subdomain, k)
__global__ void rtf_kernel(DevPlan P, int nsub, const double* R, const double* f, double* e) {
  const int lane = threadIdx.x & 31;
  for (int wk = (blockIdx.x * blockDim.x + threadIdx.x) / 32; wk < nsub * 6; wk += gridDim.x * blockDim.x / 32) {
    const int si = wk / 6, k = wk % 6;
    const SubInfo& S = P.sub[si];
    if (k >= S.d) continue;
    double acc = 0.0;
    for (int i = lane; i < S.n; i += 32) acc += R[S.R + (int64_t)k * S.n + i] * f[S.dof + i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) e[S.alpha0 + k] = acc;
  }
}

// c[alpha0 + k] = sum_j G6[(qcol + j) * 6 + k] x[map_j]  (G^T x), warp per (subdomain, k)
__global__ void gt_kernel(DevPlan P, int nsub, const double* G6, const double* x, double* c) {
  const int lane = threadIdx.x & 31;
  for (int wk = (blockIdx.x * blockDim.x + threadIdx.x) / 32; wk < nsub * 6; wk += gridDim.x * blockDim.x / 32) {
    const int si = wk / 6, k = wk % 6;
    const SubInfo& S = P.sub[si];
    if (k >= S.d) continue;
    double acc = 0.0;
    for (int j = lane; j < S.m; j += 32) acc += G6[(S.qcol + j) * 6 + k] * x[P.qmap[S.qcol + j]];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) c[S.alpha0 + k] = acc;
  }
}

// out[l] = (x ? x[l] : 0) - sgn * (G z)[l]
__global__ void gz_kernel(DevPlan P, const int* colsub, const int* c0, const int* c1, int nlam, const double* G6,
                          const double* x, const double* z, double sgn, double* out) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlam; l += gridDim.x * blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int g = e == 0 ? c0[l] : c1[l];
      if (g < 0) continue;
      const SubInfo& S = P.sub[colsub[g]];
      for (int k = 0; k < S.d; ++k) s += G6[(int64_t)g * 6 + k] * z[S.alpha0 + k];
    }
    out[l] = (x ? x[l] : 0.0) - sgn * s;
  }
}

// G^T G block (i, k) from the multiplier pairs shared by subdomains i and k
__global__ void gtg_kernel(const int4* pairs, int npairs, const int2* plist, const double* G6, double* A, int D) {
  for (int pi = blockIdx.x; pi < npairs; pi += gridDim.x) {
    const int4 pr = pairs[pi];  // x = offset_i, y = offset_k, z = list begin, w = list end
    const int a = threadIdx.x / 6, b = threadIdx.x % 6;
    if (threadIdx.x >= 36) continue;
    const int di = (pr.x >> 24) & 0xff, dk = (pr.y >> 24) & 0xff;
    const int oi = pr.x & 0xffffff, ok = pr.y & 0xffffff;
    if (a >= di || b >= dk) continue;
    double s = 0.0;
    for (int t = pr.z; t < pr.w; ++t) s += G6[(int64_t)plist[t].x * 6 + a] * G6[(int64_t)plist[t].y * 6 + b];
    A[(int64_t)(oi + a) * D + ok + b] = s;
    if (oi != ok) A[(int64_t)(ok + b) * D + oi + a] = s;
  }
}

// ---------------------------------------------------------------- dense FP64 tiles

// C = beta C + alpha op(A) op(B), row-major, 64 x 64 tile per CTA.
// lower: only tiles/entries with col <= row.  ktri: the K sum starts at
// max(row tile, col tile) (op(A) = W^T, op(B) = W with W lower triangular).
__global__ void __launch_bounds__(256) gemm64_kernel(int M, int N, int K, double alpha, const double* A, int lda,
                                                     int ta, const double* B, int ldb, int tb, double beta,
                                                     double* C, int ldc, int lower, int ktri) {
  __shared__ double As[16][kT + 1];
  __shared__ double Bs[16][kT + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int r0 = blockIdx.y * kT, c0 = blockIdx.x * kT;
  if (lower && c0 > r0 + kT - 1) return;
  double acc[4][4] = {};
  int kstart = ktri ? (max(r0, c0) / 16) * 16 : 0;
  for (int k0 = kstart; k0 < K; k0 += 16) {
    for (int idx = tid; idx < 16 * kT; idx += 256) {
      const int k = idx / kT, x = idx % kT;
      const int gi = r0 + x, gk = k0 + k, gj = c0 + x;
      As[k][x] = (gi < M && gk < K) ? (ta ? A[(int64_t)gk * lda + gi] : A[(int64_t)gi * lda + gk]) : 0.0;
      Bs[k][x] = (gj < N && gk < K) ? (tb ? B[(int64_t)gj * ldb + gk] : B[(int64_t)gk * ldb + gj]) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[k][ty + 16 * u];
        b[u] = Bs[k][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = r0 + ty + 16 * u;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = c0 + tx + 16 * v;
      if (i < M && j < N && (!lower || j <= i)) {
        double* pc = C + (int64_t)i * ldc + j;
        *pc = (beta == 0.0 ? 0.0 : beta * *pc) + alpha * acc[u][v];
      }
    }
  }
}

// Cholesky of the n x n (n <= 64) diagonal block at A (row-major, ld lda),
// in place (lower, upper part zeroed), and the inverse of the factor into
// Dinv (64 x 64, row-major, ld 64).
__global__ void __launch_bounds__(256) potrf64_kernel(double* A, int lda, int n, double* Dinv, int* status) {
  __shared__ double a[kT][kT + 1];
  __shared__ double b[kT][kT + 1];
  __shared__ double rinv[kT];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kT * kT; idx += 256) {
    const int i = idx / kT, j = idx % kT;
    a[i][j] = (i < n && j < n && j <= i) ? A[(int64_t)i * lda + j] : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      double d = a[k][k];
      if (!(d > 0.0)) {
        atomicOr(status, kStatNotSPD);
        d = 1.0;
      }
      d = sqrt(d);
      a[k][k] = d;
      rinv[k] = 1.0 / d;
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < n; i += 256) a[i][k] *= rinv[k];
    __syncthreads();
    const int rem = n - k - 1;
    for (int idx = tid; idx < rem * rem; idx += 256) {
      const int i = k + 1 + idx / rem, j = k + 1 + idx % rem;
      if (j <= i) a[i][j] -= a[i][k] * a[j][k];
    }
    __syncthreads();
  }
  // inverse of the factor, column j by thread j
  if (tid < kT) {
    const int j = tid;
    for (int i = 0; i < kT; ++i) b[i][j] = 0.0;
    if (j < n) {
      b[j][j] = rinv[j];
      for (int i = j + 1; i < n; ++i) {
        double s = 0.0;
        for (int k = j; k < i; ++k) s += a[i][k] * b[k][j];
        b[i][j] = -s * rinv[i];
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < kT * kT; idx += 256) {
    const int i = idx / kT, j = idx % kT;
    if (i < n && j < n) A[(int64_t)i * lda + j] = j <= i ? a[i][j] : 0.0;
    Dinv[i * kT + j] = b[i][j];
  }
}

__global__ void copy2d_kernel(const double* src, int lds, double* dst, int ldd, int rows, int cols, double scale) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < (int64_t)rows * cols; g += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(g / cols), j = (int)(g % cols);
    dst[(int64_t)i * ldd + j] = scale * src[(int64_t)i * lds + j];
  }
}

// ---------------------------------------------------------------- vectors

// r = d - q
__global__ void sub_kernel(const double* d, const double* q, double* r, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) r[i] = d[i] - q[i];
}

// u_i += R_i alpha_i
__global__ void add_Ralpha_kernel(DevPlan P, const int* dofsub, int64_t ndof, const double* R, const double* alpha,
                                  double* u) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ndof; g += (int64_t)gridDim.x * blockDim.x) {
    const SubInfo& S = P.sub[dofsub[g]];
    const int i = (int)(g - S.dof);
    double s = 0.0;
    for (int k = 0; k < S.d; ++k) s += R[S.R + (int64_t)k * S.n + i] * alpha[S.alpha0 + k];
    u[g] += s;
  }
}

// z = A c (D x D row-major), warp per row
__global__ void gemv_kernel(const double* A, const double* c, double* z, int D, double alpha) {
  const int lane = threadIdx.x & 31;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) / 32; row < D; row += gridDim.x * blockDim.x / 32) {
    double acc = 0.0;
    for (int j = lane; j < D; j += 32) acc += A[(int64_t)row * D + j] * c[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) z[row] = alpha * acc;
  }
}

}  // namespace

inline int grid_for(int64_t n, int per = 256, int cap = 152 * 16) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, cap));
}

size_t implicit_smem(int nmax, int maxf) { return ((size_t)nmax + maxf + (kThreads / 32) * kWF) * 8; }

void launch_implicit(int mode, const DevPlan& P, const int* order, int nsub, int* queue, const double* p,
                     const double* f, double* qi, double* u, double* uws, int64_t ustride, int nmax, int maxf,
                     int grid, size_t smem, cudaStream_t st) {
  if (mode == 3) {
    cudaFuncSetAttribute(implicit_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    implicit_kernel<3><<<grid, kThreads, smem, st>>>(P, order, nsub, queue, p, f, qi, u, uws, ustride, nmax,
                                                        maxf);
  } else if (mode == 0) {
    cudaFuncSetAttribute(implicit_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    implicit_kernel<0><<<grid, kThreads, smem, st>>>(P, order, nsub, queue, p, f, qi, u, uws, ustride, nmax,
                                                        maxf);
  } else if (mode == 1) {
    cudaFuncSetAttribute(implicit_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    implicit_kernel<1><<<grid, kThreads, smem, st>>>(P, order, nsub, queue, p, f, qi, u, uws, ustride, nmax,
                                                        maxf);
  } else {
    cudaFuncSetAttribute(implicit_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    implicit_kernel<2><<<grid, kThreads, smem, st>>>(P, order, nsub, queue, p, f, qi, u, uws, ustride, nmax,
                                                        maxf);
  }
}

void launch_unit_scale(const DevPlan& P, int nsub, double* d2, cudaStream_t st) {
  unit_scale_kernel<<<std::min(nsub, 152 * 8), 256, 0, st>>>(P, nsub, d2);
}

int implicit_occupancy(size_t smem) {
  int nb = 0;
  cudaFuncSetAttribute(implicit_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, implicit_kernel<0>, kThreads, smem);
  return std::max(nb, 1);
}

void launch_gather_minus_c(const int* c0, const int* c1, int nlam, const double* qi, const double* c, double* q,
                           cudaStream_t st) {
  gather_minus_c_kernel<<<grid_for(nlam), 256, 0, st>>>(c0, c1, nlam, qi, c, q);
}

void launch_build_G(const DevPlan& P, const int* colsub, int64_t ncols, const double* R, double* G6,
                    cudaStream_t st) {
  build_G_kernel<<<grid_for(ncols), 256, 0, st>>>(P, colsub, ncols, R, G6);
}

void launch_rtf(const DevPlan& P, int nsub, const double* R, const double* f, double* e, cudaStream_t st) {
  rtf_kernel<<<grid_for((int64_t)nsub * 6 * 32), 256, 0, st>>>(P, nsub, R, f, e);
}

void launch_gt(const DevPlan& P, int nsub, const double* G6, const double* x, double* c, cudaStream_t st) {
  gt_kernel<<<grid_for((int64_t)nsub * 6 * 32), 256, 0, st>>>(P, nsub, G6, x, c);
}

void launch_gz(const DevPlan& P, const int* colsub, const int* c0, const int* c1, int nlam, const double* G6,
               const double* x, const double* z, double sgn, double* out, cudaStream_t st) {
  gz_kernel<<<grid_for(nlam), 256, 0, st>>>(P, colsub, c0, c1, nlam, G6, x, z, sgn, out);
}

void launch_gtg(const int4* pairs, int npairs, const int2* plist, const double* G6, double* A, int D,
                cudaStream_t st) {
  if (npairs > 0) gtg_kernel<<<std::min(npairs, 152 * 32), 64, 0, st>>>(pairs, npairs, plist, G6, A, D);
}

void launch_gemm64(int M, int N, int K, double alpha, const double* A, int lda, int ta, const double* B, int ldb,
                   int tb, double beta, double* C, int ldc, int lower, int ktri, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((N + kT - 1) / kT, (M + kT - 1) / kT);
  gemm64_kernel<<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, lower, ktri);
}

void launch_potrf64(double* A, int lda, int n, double* Dinv, int* status, cudaStream_t st) {
  potrf64_kernel<<<1, 256, 0, st>>>(A, lda, n, Dinv, status);
}

void launch_copy2d(const double* src, int lds, double* dst, int ldd, int rows, int cols, double scale,
                   cudaStream_t st) {
  if (rows > 0 && cols > 0)
    copy2d_kernel<<<grid_for((int64_t)rows * cols), 256, 0, st>>>(src, lds, dst, ldd, rows, cols, scale);
}

void launch_sub(const double* d, const double* q, double* r, int n, cudaStream_t st) {
  sub_kernel<<<grid_for(n), 256, 0, st>>>(d, q, r, n);
}

void launch_add_Ralpha(const DevPlan& P, const int* dofsub, int64_t ndof, const double* R, const double* alpha,
                       double* u, cudaStream_t st) {
  add_Ralpha_kernel<<<grid_for(ndof), 256, 0, st>>>(P, dofsub, ndof, R, alpha, u);
}

void launch_gemv(const double* A, const double* c, double* z, int D, double alpha, cudaStream_t st) {
  if (D > 0) gemv_kernel<<<grid_for((int64_t)D * 32), 256, 0, st>>>(A, c, z, D, alpha);
}

}  // namespace feti
