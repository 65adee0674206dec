// Numeric factorisation K_reg,i = L_i L_i^T and the pruned forward solve
// X_i = L_i^{-1} P_i B_i^T (paper Sec. III, eq. 12; Sec. IV SYRK path).
//
// Both run as persistent kernels: each CTA pops subdomains from a queue
// sorted by decreasing cost and walks that subdomain's supernodes in
// postorder with a multifrontal scheme.  A supernode's front is
//   [ L_ss        ]  w columns (kept as the L panel, column-major f x w)
//   [ L_rs | U_s  ]  r x r update block passed to the parent (extend-add).
// For the solve, the front of supernode s holds the right-hand-side columns
// J_s = the B columns whose first nonzero row lies in s's subtree; column j
// of P B^T has one signed unit at row s_j, so column j is zero above s_j and
// only the supernodes on the path from s_j to the root touch it (pruning).
#include <cmath>

#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "symbolic.h"
#include "tc_common.cuh"

namespace feti {
namespace {

__device__ __forceinline__ int pop_item(int* queue) {
  __shared__ int item;
  __syncthreads();
  if (threadIdx.x == 0) item = atomicAdd(queue, 1);
  __syncthreads();
  return item;
}

// acc[u][v] += sum_k A[k][r0 + 16u] * B[k][c0 + 16v] for u < NU, v < NV
// (skipping v > u on diagonal tiles).  NU / NV are warp-uniform counts of
// micro-rows / micro-columns that hold real data, so padded parts of small
// fronts issue no FP64 work.
template <typename T, int NU, int NV, bool DIAG>
__device__ __forceinline__ void tile_mma_g(const T (*A)[kT], const T (*B)[kT], int kc, T acc[4][4], int r0,
                                           int c0) {
  for (int k = 0; k < kc; ++k) {
    T a[NU], b[NV];
#pragma unroll
    for (int u = 0; u < NU; ++u) a[u] = A[k][r0 + 16 * u];
#pragma unroll
    for (int v = 0; v < NV; ++v) b[v] = B[k][c0 + 16 * v];
#pragma unroll
    for (int u = 0; u < NU; ++u)
#pragma unroll
      for (int v = 0; v < NV; ++v)
        if (!DIAG || v <= u) acc[u][v] = fma(a[u], b[v], acc[u][v]);
  }
}

template <typename T, bool DIAG>
__device__ __forceinline__ void tile_mma_dispatch(const T (*A)[kT], const T (*B)[kT], int kc, T acc[4][4], int r0,
                                                  int c0, int nu, int nv) {
#define FETI_TM(U, V) \
  case (U) * 8 + (V): tile_mma_g<T, U, V, DIAG>(A, B, kc, acc, r0, c0); break;
  switch (nu * 8 + nv) {
    FETI_TM(1, 1) FETI_TM(1, 2) FETI_TM(1, 3) FETI_TM(1, 4)
    FETI_TM(2, 1) FETI_TM(2, 2) FETI_TM(2, 3) FETI_TM(2, 4)
    FETI_TM(3, 1) FETI_TM(3, 2) FETI_TM(3, 3) FETI_TM(3, 4)
    FETI_TM(4, 1) FETI_TM(4, 2) FETI_TM(4, 3) FETI_TM(4, 4)
    default: break;
  }
#undef FETI_TM
}

__device__ __forceinline__ int groups16(int valid) { return valid <= 0 ? 0 : min(4, (valid + 15) / 16); }

struct Smem {
  double D[kNB][kNB + 1];  // diagonal block, becomes L_bb
  double A[kNB][kT];
  double B[kNB][kT];       // also holds L_bb^{-1} (as [kNB][kNB + 1]) in the solve kernel
  double dinv[kNB];
  double red[kThreads / 32];
};

// Warp-level Cholesky of the nbk x nbk block D (lower, in place) with
// reciprocal pivots kept in dinv.  A non-positive pivot sets *bad and is
// replaced by 1 so the sweep finishes with finite values.
template <typename T>
__device__ void warp_chol(T (*D)[kNB + 1], T* dinv, int nbk, int* bad) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < nbk; ++k) {
    if (lane == k) {
      T d = D[k][k];
      if (!(d > (T)0)) {
        if (bad) *bad = 1;
        d = (T)1;
      }
      const T rs = rsqrt(d);  // pivot d / sqrt(d) and its reciprocal from one FP64 sequence
      D[k][k] = d * rs;
      dinv[k] = rs;
    }
    __syncwarp();
    if (lane > k && lane < nbk) D[lane][k] *= dinv[k];
    __syncwarp();
    if (lane > k && lane < nbk) {
      const T lik = D[lane][k];
      for (int j = k + 1; j <= lane; ++j) D[lane][j] -= lik * D[j][k];
    }
    __syncwarp();
  }
}

// Warp-level inverse of the lower-triangular nbk x nbk factor in D (with
// reciprocal pivots dinv): lane j computes column j of L^{-1} into Di.
template <typename T>
__device__ void warp_tri_inverse(const T (*D)[kNB + 1], const T* dinv, T (*Di)[kNB + 1], int nbk) {
  const int j = threadIdx.x & 31;
  for (int i = 0; i < kNB; ++i) Di[i][j] = (T)0;
  if (j < nbk) {
    Di[j][j] = dinv[j];
    for (int i = j + 1; i < nbk; ++i) {
      T s = (T)0;
      for (int k = j; k < i; ++k) s = fma(D[i][k], Di[k][j], s);
      Di[i][j] = -s * dinv[i];
    }
  }
  __syncwarp();
}

// Partial dense factorisation of one front: eliminate the first w columns of
// the (w+r) x (w+r) symmetric front held as Ls (column-major f x w) and W
// (column-major r x r, lower part used).  With a column range: eliminate the
// columns [kB, kE) only and apply their updates to the columns below ce only
// (the tensor-core Cholesky updates the rest itself).
__device__ void factor_front(Smem& sm, double* Ls, int f, int w, double* W, int r, int* bad, int kB = 0,
                             int kE = -1, int ce = -1) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16, warp = tid / 32;
  if (kE < 0) kE = w;
  if (ce < 0) ce = f;
  for (int kb = kB; kb < kE; kb += kNB) {
    const int nbk = min(kNB, kE - kb);
    for (int idx = tid; idx < kNB * kNB; idx += kThreads) {
      int i = idx % kNB, j = idx / kNB;
      sm.D[i][j] = (i < nbk && j <= i) ? Ls[(int64_t)(kb + j) * f + kb + i] : 0.0;
    }
    __syncthreads();
    if (warp == 0) warp_chol<double>(sm.D, sm.dinv, nbk, bad);
    __syncthreads();
    for (int idx = tid; idx < nbk * nbk; idx += kThreads) {
      int i = idx % nbk, j = idx / nbk;
      if (i >= j) Ls[(int64_t)(kb + j) * f + kb + i] = sm.D[i][j];
    }
    // panel: the rows below the block solve x L_bb^T = a, i.e. x = L_bb^{-1} a per row, with L_bb^{-1} formed
    // once by warp 0: 64 rows at a time, each row's 32 outputs split over four threads (8 each), so that all
    // threads work and no thread runs a dependent substitution chain
    auto Di = reinterpret_cast<double (*)[kNB + 1]>(&sm.B[0][0]);
    if (warp == 0) warp_tri_inverse<double>(sm.D, sm.dinv, Di, nbk);
    const int i0 = kb + nbk;
    for (int ri = i0; ri < f; ri += kT) {
      for (int idx = tid; idx < nbk * kT; idx += kThreads) {
        int xx = idx % kT, k = idx / kT;
        sm.A[k][xx] = (ri + xx < f) ? Ls[(int64_t)(kb + k) * f + ri + xx] : 0.0;
      }
      __syncthreads();
      {
        const int xx = tid % kT, jg = tid / kT;
        if (ri + xx < f && jg * 8 < nbk) {
          double acc[8] = {};
          for (int k = 0; k <= min(nbk - 1, jg * 8 + 7); ++k) {
            const double a = sm.A[k][xx];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) acc[jj] = fma(Di[jg * 8 + jj][k], a, acc[jj]);
          }
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
            if (jg * 8 + jj < nbk) Ls[(int64_t)(kb + jg * 8 + jj) * f + ri + xx] = acc[jj];
        }
      }
      __syncthreads();
    }
    // trailing update C -= L_ib L_jb^T on the lower triangle of rows/cols [i0, f)
    const int nr = f - i0;
    const int T = (nr + kT - 1) / kT;
    for (int ti = 0; ti < T; ++ti) {
      for (int tj = 0; tj <= ti; ++tj) {
        const int ri = i0 + ti * kT, cj = i0 + tj * kT;
        if (cj >= ce) break;
        for (int idx = tid; idx < nbk * kT; idx += kThreads) {
          int x = idx % kT, k = idx / kT;
          const double* col = Ls + (int64_t)(kb + k) * f;
          sm.A[k][x] = (ri + x < f) ? col[ri + x] : 0.0;
          sm.B[k][x] = (cj + x < f) ? col[cj + x] : 0.0;
        }
        __syncthreads();
        double acc[4][4] = {};
        const int nu = groups16(f - ri - 2 * warp), nv = groups16(f - cj);
        if (ti == tj) tile_mma_dispatch<double, true>(sm.A, sm.B, nbk, acc, ty, tx, nu, nv);
        else tile_mma_dispatch<double, false>(sm.A, sm.B, nbk, acc, ty, tx, nu, nv);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          int i = ri + ty + 16 * u;
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            int j = cj + tx + 16 * v;
            if (u < nu && v < nv && i < f && j <= i && j < ce) {
              double* p = (j < w) ? Ls + (int64_t)j * f + i : W + (int64_t)(j - w) * r + (i - w);
              *p -= acc[u][v];
            }
          }
        }
        __syncthreads();
      }
    }
  }
}

// ---------------------------------------------------------------- packed fronts in shared memory
//
// A front of width f <= kMidFront is assembled as a packed lower triangle
// (column-major: column k holds rows k .. f-1) in shared memory, its first w
// columns are factored right-looking, and the team (one warp, or the whole
// CTA) spreads each trailing update evenly over its threads, so no FP64 work
// is spent on padding.  Entry (i, k), i >= k, sits at pidx(f, i, k).

constexpr int kWarpSlot = kSmallFront * (kSmallFront + 1) / 2;           // doubles per warp
constexpr int kFrontSmem = (8 * kWarpSlot > kMidFront * (kMidFront + 1) / 2 ? 8 * kWarpSlot
                                                                            : kMidFront * (kMidFront + 1) / 2);
static_assert(kThreads == 256, "the small-front phase assumes 8 warps per CTA");
static_assert(sizeof(Smem) <= (size_t)kFrontSmem * 8, "the tiled path aliases the packed-front buffer");

__device__ __forceinline__ int pidx(int f, int i, int k) { return k * f - (k * (k - 1)) / 2 + (i - k); }

template <int TEAM>
__device__ __forceinline__ void team_sync() {
  if constexpr (TEAM == 32) __syncwarp();
  else __syncthreads();
}

// Update block of child gc: a small child's lives in the CTA's small region, a split root's (a child factored
// by another task) in its hand-over slot, others on the stack.
__device__ __forceinline__ const double* child_update(const DevPlan& P, int gc, const double* stack,
                                                      const double* smallreg, const double* hand) {
  if (hand && P.sn_hoff[gc] >= 0) return hand + P.sn_hoff[gc];
  return P.sn_small[gc] ? smallreg + P.usm_ofs[gc] : stack + P.upd_ofs[gc];
}

// Assemble front gs (K entries, rho on fixing DOFs, children's update blocks),
// factor its first w columns, store the f x w panel to L (zeros above the
// diagonal) and, if Uout, the r x r update block (column-major) for the parent.
template <int TEAM>
__device__ void packed_front(const DevPlan& P, const SubInfo& S, int s, const double* K, double* L, double rho,
                             double* Fp, const double* stack, const double* smallreg, double* Uout, int* bad,
                             int tid, bool factor = true, const double* hand = nullptr) {
  const int gs = S.sn0 + s;
  const int w = P.sn_w[gs], r = P.sn_r[gs], f = w + r;
  const int np = f * (f + 1) / 2;
  const int64_t L0 = P.Lofs[gs];
  for (int e = tid; e < np; e += TEAM) Fp[e] = 0.0;
  team_sync<TEAM>();
  for (int64_t kk = P.kmap_off[gs] + tid; kk < P.kmap_off[gs + 1]; kk += TEAM) {
    const int64_t rel = P.kmap_dst[kk] - L0;  // column-major f x w panel position
    Fp[pidx(f, (int)(rel % f), (int)(rel / f))] = K[P.kmap_src[kk]];
  }
  team_sync<TEAM>();
  for (int k = tid; k < S.nfix; k += TEAM)
    if (P.fix_sn[S.fix0 + k] == s) {
      const int64_t rel = P.fix_pos[S.fix0 + k] - L0;
      Fp[pidx(f, (int)(rel % f), (int)(rel / f))] += rho;
    }
  for (int c = P.ch_off[gs]; c < P.ch_off[gs + 1]; ++c) {
    const int gc = S.sn0 + P.ch_list[c];
    const int rc = P.sn_r[gc];
    const double* U = child_update(P, gc, stack, smallreg, hand);
    const int* rl = P.rel + P.rel_off[gc];
    team_sync<TEAM>();
    for (int b = 0; b < rc; ++b)
      for (int a = b + tid; a < rc; a += TEAM) Fp[pidx(f, rl[a], rl[b])] += __ldcg(U + (int64_t)b * rc + a);
  }
  team_sync<TEAM>();
  // blocked right-looking partial factorisation of the first w columns: one warp
  // factors kPB columns (warp syncs only), then the whole team applies their
  // rank-kPB update to the trailing triangle, kPB FMAs per element
  constexpr int kPB = 8;
  const int lane = tid & 31;
  for (int j0 = 0; factor && j0 < w; j0 += kPB) {
    const int jb = min(kPB, w - j0);
    if (tid < 32) {
      for (int j = j0; j < j0 + jb; ++j) {
        const int cj = pidx(f, j, j);
        // one reciprocal square root by lane 0 gives both the pivot (pv / sqrt(pv)) and the column scale, so
        // the warp spends one FP64 sequence per column instead of a square root plus a division on every lane
        // (this GPU's FP64 pipe is narrow and the small fronts have short columns)
        double rs = 0.0;
        if (lane == 0) {
          double pv = Fp[cj];
          if (!(pv > 0.0)) {
            *bad = 1;
            pv = 1.0;
          }
          rs = rsqrt(pv);
          Fp[cj] = pv * rs;
        }
        const double inv = __shfl_sync(0xffffffffu, rs, 0);
        __syncwarp();
        for (int i = j + 1 + lane; i < f; i += 32) Fp[cj + (i - j)] *= inv;
        __syncwarp();
        // update the panel's later columns k in (j, j0 + jb), rows i >= k
        for (int k = j + 1; k < j0 + jb; ++k) {
          const double lkj = Fp[cj + (k - j)];
          const int pk = pidx(f, k, k);
          for (int i = k + lane; i < f; i += 32) Fp[pk + (i - k)] = fma(-Fp[cj + (i - j)], lkj, Fp[pk + (i - k)]);
        }
        __syncwarp();
      }
    }
    team_sync<TEAM>();
    // trailing update A[i][k] -= sum_{j in panel} L[i][j] L[k][j], k >= j0 + jb, i >= k:
    // element e of the packed trailing triangle goes to thread e mod TEAM
    const int k0 = j0 + jb;
    int k = k0, rem = tid;
    while (k < f && rem >= f - k) {
      rem -= f - k;
      ++k;
    }
    while (k < f) {
      const int i = k + rem;
      double acc = Fp[pidx(f, i, k)];
#pragma unroll
      for (int u = 0; u < kPB; ++u) {
        if (u < jb) {
          const int cj = pidx(f, j0 + u, j0 + u);
          acc = fma(-Fp[cj + (i - j0 - u)], Fp[cj + (k - j0 - u)], acc);
        }
      }
      Fp[pidx(f, i, k)] = acc;
      rem += TEAM;
      while (k < f && rem >= f - k) {
        rem -= f - k;
        ++k;
      }
    }
    team_sync<TEAM>();
  }
  for (int idx = tid; idx < f * w; idx += TEAM) {
    const int row = idx % f, col = idx / f;
    L[L0 + idx] = row >= col ? Fp[pidx(f, row, col)] : 0.0;
  }
  if (Uout)
    for (int idx = tid; idx < r * r; idx += TEAM) {
      const int a = idx % r, b = idx / r;
      Uout[idx] = a >= b ? Fp[pidx(f, w + a, w + b)] : 0.0;
    }
  team_sync<TEAM>();
}

// Assemble a front of the tiled path in global memory: the f x w panel Ls (column-major, in the factor's
// storage) and the r x r bottom block W, from the K entries, the fixing-DOF penalty rho and the children's update
// blocks (stack, small region or hand-over slot).
__device__ void assemble_tiled(const DevPlan& P, const SubInfo& S, int s, const double* K, double* L, double rho,
                               double* W, const double* stack, const double* smallreg, const double* hand) {
  const int tid = threadIdx.x;
  const int gs = S.sn0 + s;
  const int w = P.sn_w[gs], r = P.sn_r[gs], f = w + r;
  double* Ls = L + P.Lofs[gs];
  for (int64_t idx = tid; idx < (int64_t)f * w; idx += kThreads) Ls[idx] = 0.0;
  for (int64_t idx = tid; idx < (int64_t)r * r; idx += kThreads) W[idx] = 0.0;
  __syncthreads();
  for (int64_t k = P.kmap_off[gs] + tid; k < P.kmap_off[gs + 1]; k += kThreads)
    L[P.kmap_dst[k]] = K[P.kmap_src[k]];
  __syncthreads();
  for (int k = tid; k < S.nfix; k += kThreads)
    if (P.fix_sn[S.fix0 + k] == s) L[P.fix_pos[S.fix0 + k]] += rho;
  for (int c = P.ch_off[gs]; c < P.ch_off[gs + 1]; ++c) {
    const int gc = S.sn0 + P.ch_list[c];
    const int rc = P.sn_r[gc];
    const double* U = child_update(P, gc, stack, smallreg, hand);
    const int* rl = P.rel + P.rel_off[gc];
    __syncthreads();
    // four elements per thread and step, their loads issued before their read-modify-writes (distinct
    // targets: rel is one-to-one)
    const int64_t n = (int64_t)rc * rc;
    for (int64_t base = tid; base < n; base += 4 * kThreads) {
      double* dst[4];
      double v[4], cur[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t idx = base + (int64_t)u * kThreads;
        dst[u] = nullptr;
        if (idx < n) {
          const int b = (int)(idx / rc), a = (int)(idx - (int64_t)b * rc);
          if (a >= b) {
            const int ra = rl[a], rb = rl[b];
            v[u] = __ldcg(U + idx);
            dst[u] = rb < w ? Ls + (int64_t)rb * f + ra : W + (int64_t)(rb - w) * r + (ra - w);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) cur[u] = dst[u] ? *dst[u] : 0.0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (dst[u]) *dst[u] = cur[u] + v[u];
    }
  }
}

// One CTA per subdomain (persistent, queue sorted by decreasing cost).
// Phase 1: the small subtrees, level by level from the leaves, one warp per
// front.  Phase 2: the remaining supernodes in postorder, fronts up to
// kMidFront in shared memory across the CTA, larger ones by the tiled path.
// flags: kCholNoReg factors K itself (no fixing-DOF penalty); kCholStopRoot
// assembles the last (root) supernode's front but does not eliminate it, so
// with the DOFs B touches ordered last the root panel holds the Schur
// complement of the interior onto them (lower triangle, column-major).
// Work items (subdomain, task, global task id, parent's global task id).  use_tasks = 0: an item is a whole
// subdomain.  use_tasks = 1: an item is one task of the plan's split (plan_tasks): it factors only the
// supernodes of that task, first waiting (bounded) until its child tasks have finished (they precede it in
// the item list, so they have been taken by running CTAs), reads the update blocks of split children from
// their hand-over slots, writes its own root's there when that root is split, and counts itself done at its
// parent task.
__global__ void __launch_bounds__(kThreads, 4) chol_kernel(DevPlan P, const int4* items, int nitems, int use_tasks,
                                                         int* queue, int* tdone, double* hand_all, double* ws,
                                                         int64_t ws_stride, int64_t front_sz, int64_t stack_sz,
                                                         int flags, int* status) {
  extern __shared__ double dsm[];
  Smem& sm = *reinterpret_cast<Smem*>(dsm);
  __shared__ int bad;
  __shared__ double red[kThreads / 32];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  double* W = ws + (int64_t)blockIdx.x * ws_stride;
  double* stack = W + front_sz;
  double* smallreg = stack + stack_sz;
  for (;;) {
    int it = pop_item(queue);
    if (it >= nitems) return;
    const int4 item = items[it];
    const int si = item.x, task = item.y;
    const SubInfo S = P.sub[si];
    const double* K = P.Kval + S.Kval;
    double* L = P.L + S.L;
    double* hand = hand_all + S.hbase;  // hand-over slots of split roots (also when one CTA takes the subdomain)
    if (use_tasks && P.task_nchild[item.z] > 0) {
      // the child tasks were taken before this one and are running: wait for them (bounded)
      if (tid == 0) {
        int ok = 0;
        for (int i = 0; i < (1 << 26); ++i) {
          if (*(volatile int*)(tdone + item.z) >= P.task_nchild[item.z]) {
            ok = 1;
            break;
          }
          __nanosleep(64);
        }
        if (!ok) atomicOr(status, kStatTimeout);
        __threadfence();
        bad = ok ? 0 : 2;
        // given up (status set): still count this task done at its parent, so that a failure does not make
        // every ancestor wait out its own limit
        if (!ok && item.w >= 0) atomicAdd(tdone + item.w, 1);
      }
      __syncthreads();
      if (bad == 2) continue;
    }
    __syncthreads();
    if (tid == 0) bad = 0;
    // rho = max diag K_i (fixing-node penalty)
    double mx = 0.0;
    for (int i = tid; i < S.n; i += kThreads) mx = fmax(mx, K[P.diag_src[S.diag0 + i]]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    double rho = red[0];
    for (int k = 1; k < kThreads / 32; ++k) rho = fmax(rho, red[k]);
    if (tid == 0) P.rho[si] = rho;
    if (flags & kCholNoReg) rho = 0.0;
    // phase 1: small subtrees, one warp per front
    const int* lvo = P.lvl_off + S.lvl0;
    double* Fw = dsm + warp * kWarpSlot;
    for (int l = 0; l < S.nlev; ++l) {
      bool any = false;
      for (int q = lvo[l]; q < lvo[l + 1]; ++q) {
        const int gq = S.sn0 + P.lvl_sn[q];
        any |= P.sn_small[gq] != 0 && (!use_tasks || P.sn_task[gq] == task);
      }
      if (!any) continue;
      for (int q = lvo[l] + warp; q < lvo[l + 1]; q += kThreads / 32) {
        const int s = P.lvl_sn[q];
        const int gs = S.sn0 + s;
        if (!P.sn_small[gs] || (use_tasks && P.sn_task[gs] != task)) continue;
        // a small subtree whose parent is factored by another task hands its update block over
        double* Uout = P.sn_parent[gs] < 0 ? nullptr
                       : P.sn_hoff[gs] >= 0 ? hand + P.sn_hoff[gs] : smallreg + P.usm_ofs[gs];
        packed_front<32>(P, S, s, K, L, rho, Fw, stack, smallreg, Uout, &bad, lane,
                         !((flags & kCholStopRoot) && s == S.nsn - 1));
      }
      __syncthreads();
    }
    // phase 2: the rest in postorder
    for (int s = 0; s < S.nsn; ++s) {
      const int gs = S.sn0 + s;
      if (P.sn_small[gs] || (use_tasks && P.sn_task[gs] != task)) continue;
      if ((flags & kCholSkipBig) && P.sn_big[gs]) continue;  // the tensor-core kernel's fronts
      const int w = P.sn_w[gs], r = P.sn_r[gs], f = w + r;
      double* Uout = P.sn_parent[gs] < 0 ? nullptr
                     : (hand && P.sn_hoff[gs] >= 0) ? hand + P.sn_hoff[gs] : stack + P.upd_ofs[gs];
      const bool factor = !((flags & kCholStopRoot) && s == S.nsn - 1);
      if (f <= kMidFront) {
        packed_front<kThreads>(P, S, s, K, L, rho, dsm, stack, smallreg, Uout, &bad, tid, factor, hand);
        continue;
      }
      double* Ls = L + P.Lofs[gs];
      assemble_tiled(P, S, s, K, L, rho, W, stack, smallreg, hand);
      __syncthreads();
      if (factor) factor_front(sm, Ls, f, w, W, r, &bad);
      __syncthreads();
      if (Uout)
        for (int64_t idx = tid; idx < (int64_t)r * r; idx += kThreads) Uout[idx] = W[idx];
      __syncthreads();
    }
    __syncthreads();
    if (tid == 0) {
      if (bad) atomicOr(status, kStatNotSPD);
      if (use_tasks && item.w >= 0) {
        __threadfence();  // this task's factor panels and hand-over block before the count
        atomicAdd(tdone + item.w, 1);
      }
    }
  }
}

// ---------------------------------------------------------------- tensor-core Cholesky of the large fronts
//
// The fronts at least big_f wide and their ancestors (the top of each supernodal tree) are factored by
// chol_tc_kernel after chol_kernel has done everything below them.  A front's w own columns go in blocks of
// 128: the block's columns are eliminated on the FP64 pipe (32-column steps, their updates applied to the
// block's own columns only), and then the trailing matrix C = front[kE:, kE:] (its lower triangle, in Ls and W)
// takes the block's rank-128 update C -= A A^T, A = Ls[kE:, kB:kE], on the tensor cores by exact slicing of
// FP64 into bf16 integers (the Ozaki scheme): each row i of A is scaled by a power of two 2^(e_i - 6) with
// e_i the largest exponent in the row, and its 63 leading fixed-point bits are cut into 9 signed 7-bit
// integers s_p (p = 0 most significant), each exact in bf16, so A_ik = 2^(e_i - 6) sum_p s_p,ik 2^(-7p) up to
// 2^(e_i - 62).  The products of slices p, q (p + q <= 8, 45 pairs) are summed over K = 128 on the tensor cores
// with FP32 accumulation, one TMEM accumulator per d = p + q <= 7 (the d = 8 products into the d = 7 one, their
// B slices scaled by 2^-7).  For d <= 6 every partial sum is an integer below (d + 1) 128 127^2 < 2^24, so those
// FP32 sums are exact; the d = 7 one lies 2^-49 below the leading scale.  The epilogue combines them,
// sum_k A_ik A_jk = 2^(e_i + e_j - 40) (sum_{d <= 4} acc_d 2^(7 (4 - d)) + sum_{d >= 5} acc_d 2^(7 (4 - d))),
// the first sum exactly in 64-bit integers, the small rest in FP32 (its rounding below 2^-53 of K sigma_i sigma_j,
// sigma = 2^(e + 1)), and applies C_ij -= that with one FP64 FMA.  The dropped pairs (p + q >= 9) and the cut
// bits add below K 2^(e_i + e_j - 58): the whole error stays below K 2^-52 sigma_i sigma_j, inside FP64's own
// normwise bound for the same dot product (tests/test_slicing_model.py checks the model on the host).
constexpr int kOzS = 9;                              // slices of 7 bits
constexpr int kOzAcc = 8;  // accumulators: d = 0 .. 6, and d = 7 with the d = 8 products (B slices scaled by 2^-7)
constexpr int kOzK = 128;                            // columns of one panel block (K of one update)
constexpr int kOzKC = 32;                            // K per stage: one 64-byte swizzled row per operand row
constexpr int kOzN = 32;                             // C tile: 128 rows x 32 columns (9 accumulators x 32 TMEM columns)
constexpr int kOzM = 128;                            // rows of a C tile (the MMA M)
constexpr int kOzOpA = kOzM * 64, kOzOpB = kOzN * 64;
constexpr int kOzStage = kOzS * (kOzOpA + 2 * kOzOpB);  // 108 KB: A slices, B slices, B slices x 2^-7 of a chunk
constexpr int kOzStages = 2;
constexpr int kOzSetCols = kOzAcc * kOzN;               // TMEM columns of one accumulator set (two sets)
constexpr int kCholTcDyn = 1024 + kOzStages * kOzStage;
static_assert(sizeof(Smem) <= kOzStages * kOzStage, "the FP64 steps' buffers alias the stage ring");

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

// Layout of the slices in the per-CTA scratch: for slice p (p >= 9: slice p - 9 times 2^-7) and 32-deep chunk c,
// the rows one after another
// (npad = rows rounded up to 128), each row 32 bf16 = 64 bytes with its four 16-byte pieces already in the
// 64-byte swizzle of an 8-row atom (piece q of row r at q ^ ((r >> 1) & 3)): any 8-row-aligned run of rows of
// one (p, c) is a ready MMA operand, loaded by one bulk copy.
__device__ __forceinline__ int64_t oz_row(int p, int c, int npad, int r) {
  return ((int64_t)(p * (kOzK / kOzKC) + c) * npad + r) * kOzKC;
}

// Slices of A = Ls[i0 + i, kb0 + k] (i < n = f - i0, k < K = ke0 - kb0 <= 128; zero for k >= K and for the
// padding rows): row exponent EX[i] and the slices in the layout above.  A warp takes 32 rows (lane = row: the
// loads of one column are contiguous).
__device__ void oz_slice(const double* Ls, int f, int i0, int kb0, int ke0, uint16_t* SL, int* EX) {
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int n = f - i0, K = ke0 - kb0, npad = (n + kOzM - 1) / kOzM * kOzM;
  const int nch = (K + kOzKC - 1) / kOzKC;  // the chunks the update reads
  for (int rb = warp * 32; rb < npad; rb += kThreads) {
    const int i = rb + lane;
    const bool ok = i < n;
    int e = -1074;
    for (int k = 0; k < K; ++k) {
      const double x = ok ? Ls[(int64_t)(kb0 + k) * f + i0 + i] : 0.0;
      const int be = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
      if (be) e = max(e, be - 1023);
    }
    if (ok) EX[i] = e;
    for (int kc = 0; kc < nch * kOzKC; kc += 8) {
      uint32_t pk[kOzS][4], pks[kOzS][4];
#pragma unroll
      for (int kk = 0; kk < 8; kk += 2) {
        int sv[2][kOzS];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = kc + kk + h;
          const double x = (ok && k < K) ? Ls[(int64_t)(kb0 + k) * f + i0 + i] : 0.0;
          const long long b = __double_as_longlong(x);
          const int be = (int)((b >> 52) & 0x7FF);
          unsigned long long F = 0;
          if (be) {
            const unsigned long long m = (unsigned long long)(b & 0xFFFFFFFFFFFFFLL) | (1ULL << 52);
            const int sh = (be - 1023) - e + 10;  // <= 10: F < 2^63
            F = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> -sh) : 0ULL);
          }
          const bool neg = b < 0;
#pragma unroll
          for (int p = 0; p < kOzS; ++p) {
            const int v = (int)((F >> (56 - 7 * p)) & 127ULL);
            sv[h][p] = neg ? -v : v;
          }
        }
#pragma unroll
        for (int p = 0; p < kOzS; ++p) {
          const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn((float)sv[0][p]));
          const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn((float)sv[1][p]));
          pk[p][kk / 2] = lo | (hi << 16);
          // the same integer times 2^-7 (exact in bf16): the B operand of the d = 8 products
          const uint32_t los = __bfloat16_as_ushort(__float2bfloat16_rn((float)sv[0][p] * 0x1p-7f));
          const uint32_t his = __bfloat16_as_ushort(__float2bfloat16_rn((float)sv[1][p] * 0x1p-7f));
          pks[p][kk / 2] = los | (his << 16);
        }
      }
      const int c = kc / kOzKC, q = (kc % kOzKC) / 8;
#pragma unroll
      for (int p = 0; p < kOzS; ++p) {
        const int64_t o = ((q ^ ((i >> 1) & 3)) * 8);
        *reinterpret_cast<uint4*>(SL + oz_row(p, c, npad, i) + o) = make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
        *reinterpret_cast<uint4*>(SL + oz_row(kOzS + p, c, npad, i) + o) =
            make_uint4(pks[p][0], pks[p][1], pks[p][2], pks[p][3]);
      }
    }
  }
}

// the row exponents follow the slices of an n-row A
__device__ __forceinline__ int* oz_ex(uint16_t* SL, int n) {
  const int npad = (n + kOzM - 1) / kOzM * kOzM;
  return reinterpret_cast<int*>(SL + oz_row(2 * kOzS, 0, npad, 0));
}

__device__ __forceinline__ void oz_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void oz_bulk(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// C -= A A^T on the lower triangle of the trailing matrix (rows [i0, f), columns [i0, ce); columns < w in Ls,
// the others in W) from the slices.  Tiles of 128 rows x 32 columns with a column block not right of the row
// block.  Warp 0 (one thread) loads each 32-deep chunk with 27 bulk copies (A slices, B slices, scaled B slices)
// completing on the stage's "full" mbarrier and, one chunk behind, issues its 45 x 2 MMAs (slice pair p, q into
// accumulator min(p + q, 7) of the tile's accumulator set: TMEM columns 256 (tile mod 2) + 32 accumulator) and
// commits them to the stage's "empty" mbarrier, and after a tile's last chunk to the set's "accumulators full"
// mbarrier.  Warps 4-7 combine the accumulators of each tile (epilogue above) while warp 0 already multiplies
// the next tile into the other set, and release the set on its "accumulators empty" mbarrier (one arrival per
// warp).  tcnt counts the CTA's tiles (the sets' phases).  Every wait is bounded.
__device__ bool oz_update(uint8_t* ring, uint64_t* gbar, uint64_t* fbar, uint64_t* afull, uint64_t* aempty,
                          uint32_t tmem, uint32_t& g, uint32_t& tcnt, int* abort_flag, const uint16_t* SL,
                          const int* EX, int n, int K, double* Ls, int f, int w, double* W, int r, int i0, int ce) {
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  volatile int* abortv = abort_flag;
  const int ntm = (n + kOzM - 1) / kOzM, npad = ntm * kOzM;
  const int nce = ce - i0;               // columns of C
  constexpr int kTnPerTm = kOzM / kOzN;  // column blocks per row block
  int ntile = 0;  // tiles (tm, tn) with a column block not right of the row block: tn < (tm + 1) kTnPerTm
  const int ntnmax = (nce + kOzN - 1) / kOzN;
  for (int tm = 0; tm < ntm; ++tm) ntile += min((tm + 1) * kTnPerTm, ntnmax);
  const int nck = (K + kOzKC - 1) / kOzKC;
  const int total = ntile * nck;
  if (total == 0) return true;
  const uint32_t sb0 = smem_u32(ring);
  const uint32_t g0 = g, t0 = tcnt;
  constexpr uint32_t idesc = idesc_m128(1u, (uint32_t)kOzN);
  auto tile_of = [&](int t, int& tm, int& tn) {
    tm = 0;
    for (;;) {
      const int c = min((tm + 1) * kTnPerTm, ntnmax);
      if (t < c) break;
      t -= c;
      ++tm;
    }
    tn = t;
  };
  __syncthreads();  // the slices are written and the ring's earlier generic use is over
  if (warp == 0) {
    if (lane == 0) {
      int last_load = -1, last_mma = -1;
      auto load = [&](int q) {  // the 27 bulk copies of chunk q into its stage
        last_load = q;
        const uint32_t st = (g0 + q) % kOzStages, sbase = sb0 + st * kOzStage;
        const uint32_t full = smem_u32(&fbar[st]);
        const int ck = q % nck;
        int tm, tn;
        tile_of(q / nck, tm, tn);
        oz_expect(full, (uint32_t)kOzStage);
#pragma unroll 1
        for (int p = 0; p < kOzS; ++p) {
          oz_bulk(sbase + p * kOzOpA, SL + oz_row(p, ck, npad, tm * kOzM), kOzOpA, full);
          oz_bulk(sbase + kOzS * kOzOpA + p * kOzOpB, SL + oz_row(p, ck, npad, tn * kOzN), kOzOpB, full);
          oz_bulk(sbase + kOzS * (kOzOpA + kOzOpB) + p * kOzOpB, SL + oz_row(kOzS + p, ck, npad, tn * kOzN), kOzOpB,
                  full);
        }
      };
      asm volatile("fence.proxy.async.global;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bool ok = true;
      load(0);
      for (int j = 0; j < total && ok; ++j) {
        const int ck = j % nck, tile = j / nck;
        const uint32_t st = (g0 + j) % kOzStages, tg = t0 + tile, set = tg & 1;
        const int q = j + 1;  // the next chunk: its stage is free once the MMAs of the chunk that used it are done
        if (q < total) {
          if (q >= kOzStages) {
            const uint32_t gp = g0 + q - kOzStages;
            ok = mbar_wait(smem_u32(&gbar[gp % kOzStages]), (gp / kOzStages) & 1);
          }
          if (ok) load(q);
        }
        // a tile's first chunk: its accumulator set is free once the epilogue of the tile two before is done
        if (ok && ck == 0 && tg >= 2) ok = mbar_wait(smem_u32(&aempty[set]), ((tg >> 1) - 1) & 1);
        if (ok) ok = mbar_wait(smem_u32(&fbar[st]), ((g0 + j) / kOzStages) & 1);
        if (ok && *abortv) ok = false;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sA = sb0 + st * kOzStage, sB = sA + kOzS * kOzOpA, sBs = sB + kOzS * kOzOpB;
        const uint32_t acc0 = tmem + set * kOzSetCols;
#pragma unroll 1
        for (int p = 0; p < kOzS; ++p)
#pragma unroll 1
          for (int qq = 0; qq < kOzS - p; ++qq) {
            const bool d8 = p + qq == kOzAcc;  // the d = 8 pairs go into accumulator 7 with B scaled by 2^-7
            const uint32_t acc = acc0 + (uint32_t)((d8 ? kOzAcc - 1 : p + qq) * kOzN);
            const uint32_t bq = (d8 ? sBs : sB) + qq * kOzOpB;
#pragma unroll
            for (int kk = 0; kk < kOzKC / 16; ++kk)
              mma_f16(acc, sw64_desc(sA + p * kOzOpA + kk * 32), sw64_desc(bq + kk * 32), idesc,
                      (ck > 0 || p > 0 || kk > 0 || d8) ? 1u : 0u);
          }
        mma_commit(smem_u32(&gbar[st]));
        if (ck == nck - 1) mma_commit(smem_u32(&afull[set]));
        last_mma = j;
      }
      if (!ok) {
        *abortv = 1;
        // wait (bounded) for the last copies and MMAs issued
        if (last_mma >= 0) {
          const uint32_t gq = g0 + last_mma;
          mbar_wait(smem_u32(&gbar[gq % kOzStages]), (gq / kOzStages) & 1);
        }
        if (last_load > last_mma) {
          const uint32_t gq = g0 + last_load;
          mbar_wait(smem_u32(&fbar[gq % kOzStages]), (gq / kOzStages) & 1);
        }
      }
    }
    __syncwarp();
  } else if (warp >= 4) {
    const int q4 = warp % 4;  // TMEM lane quarter: rows q4 * 32 .. + 31 of the tile
    for (int tile = 0; tile < ntile; ++tile) {
      const uint32_t tg = t0 + tile, set = tg & 1;
      int ok = 1;
      if (lane == 0) ok = !*abortv && mbar_wait(smem_u32(&afull[set]), (tg >> 1) & 1);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) *abortv = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int tm, tn;
      tile_of(tile, tm, tn);
      const int ri = tm * kOzM + q4 * 32 + lane;  // row of C (relative to i0)
      const int gi = i0 + ri;
      const int ei = ri < n ? EX[ri] : 0;
#pragma unroll 1
      for (int cg = 0; cg < kOzN / 8; ++cg) {
        const int cbase = tn * kOzN + cg * 8;  // first column of this group (relative to i0)
        uint32_t a[kOzAcc][8];
#pragma unroll
        for (int d = 0; d < kOzAcc; ++d)
          tmem_ld8(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(set * kOzSetCols + d * kOzN + cg * 8), a[d]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (ri < n) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int cj = cbase + e, gj = i0 + cj;
            if (cj < nce && gj <= gi) {
              long long I = 0;
#pragma unroll
              for (int d = 0; d <= 4; ++d)
                I += (long long)__float2int_rn(__uint_as_float(a[d][e])) << (7 * (4 - d));
              float small = 0.f;  // sum_{d >= 5} acc_d 2^(-7 (d - 4)), Horner from the smallest
#pragma unroll
              for (int d = kOzAcc - 1; d >= 5; --d) small = (small + __uint_as_float(a[d][e])) * 0x1p-7f;
              const double t = (double)I + (double)small;
              const int ex = ei + EX[cj] - 40;
              const double sc = ex >= -1022 ? __longlong_as_double((long long)(ex + 1023) << 52) : 0.0;
              double* pc = gj < w ? Ls + (int64_t)gj * f + gi : W + (int64_t)(gj - w) * r + (gi - w);
              *pc = fma(-t, sc, *pc);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&aempty[set])) : "memory");
    }
  }
  __syncthreads();  // every role has finished this update
  g = g0 + total;
  tcnt = t0 + ntile;
  return !*abortv;
}

// The large fronts (P.sn_big), one task of the plan's split per item (subdomain, task, global task id, parent's
// global task id), children before parents; one CTA per SM (the stage ring takes 217 KB of shared memory and
// the two accumulator sets all 512 TMEM columns), all resident.  The fronts' children outside the set
// handed their update blocks over (chol_kernel ran first); a large child task's block comes from its hand-over
// slot after a bounded wait on the task's counter of finished large children (tdone), others through the
// CTA's stack as in chol_kernel.  The same flags as chol_kernel.
__global__ void __launch_bounds__(kThreads, 1) chol_tc_kernel(DevPlan P, const int4* items, int nitems, int* queue,
                                                            int* tdone, double* hand_all, double* ws,
                                                            int64_t ws_stride, int64_t front_sz, uint16_t* slices,
                                                            int64_t slice_stride, int flags, int* status) {
  extern __shared__ uint8_t oz_raw[];
  uint8_t* ring = oz_raw + ((1024u - (smem_u32(oz_raw) & 1023u)) & 1023u);
  Smem& sm = *reinterpret_cast<Smem*>(ring);  // the FP64 steps' buffers (never in use with the ring)
  __shared__ uint64_t gbar[kOzStages], fbar[kOzStages];  // per stage: MMAs done ("empty"), copies landed ("full")
  __shared__ uint64_t afull[2], aempty[2];  // per accumulator set: tile multiplied / epilogue done
  __shared__ uint32_t tmem_s;
  __shared__ int abort_s, bad;
  __shared__ double red[kThreads / 32];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int k = 0; k < kOzStages; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&gbar[k])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fbar[k])));
    }
    for (int k = 0; k < 2; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&afull[k])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&aempty[k])));  // the 4 epilogue warps
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_s = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_s;
  uint32_t g = 0, tcnt = 0;
  double* W = ws + (int64_t)blockIdx.x * ws_stride;
  double* stack = W + front_sz;
  uint16_t* SL = slices + (int64_t)blockIdx.x * slice_stride;
  for (;;) {
    const int it = pop_item(queue);
    if (it >= nitems) break;
    const int4 item = items[it];
    const int si = item.x, task = item.y;
    const SubInfo S = P.sub[si];
    const double* K = P.Kval + S.Kval;
    double* L = P.L + S.L;
    double* hand = hand_all + S.hbase;
    if (tid == 0) {
      bad = 0;
      // the large child tasks were taken before this one and are running: wait for them (bounded)
      int ok = 1;
      if (P.task_nbig[item.z] > 0) {
        ok = 0;
        for (int i = 0; i < (1 << 26); ++i) {
          if (*(volatile int*)(tdone + item.z) >= P.task_nbig[item.z]) {
            ok = 1;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
      if (!ok) {
        atomicOr(status, kStatTimeout);
        bad = 2;
        if (item.w >= 0) atomicAdd(tdone + item.w, 1);  // no cascade of waits above a failure
      }
    }
    __syncthreads();
    if (bad == 2) continue;
    double mx = 0.0;  // rho = max diag K_i, as in chol_kernel
    for (int i = tid; i < S.n; i += kThreads) mx = fmax(mx, K[P.diag_src[S.diag0 + i]]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    double rho = red[0];
    for (int k = 1; k < kThreads / 32; ++k) rho = fmax(rho, red[k]);
    if (flags & kCholNoReg) rho = 0.0;
    __syncthreads();
    for (int s = 0; s < S.nsn && !abort_s; ++s) {
      const int gs = S.sn0 + s;
      if (!P.sn_big[gs] || P.sn_task[gs] != task) continue;
      const int w = P.sn_w[gs], r = P.sn_r[gs], f = w + r;
      double* Ls = L + P.Lofs[gs];
      assemble_tiled(P, S, s, K, L, rho, W, stack, nullptr, hand);
      __syncthreads();
      if (!((flags & kCholStopRoot) && s == S.nsn - 1)) {
        bool okf = true;
        for (int kB = 0; kB < w && okf; kB += kOzK) {
          const int kE = min(w, kB + kOzK);
          // the block's 32-column steps: the pivot block and the panel below it on the FP64 pipe, the rank-32
          // update of the block's later columns on the tensor cores
          for (int kb = kB; kb < kE && okf; kb += kNB) {
            const int ke = min(kE, kb + kNB);
            factor_front(sm, Ls, f, w, W, r, &bad, kb, ke, ke);
            __syncthreads();
            if (ke < kE) {
              int* EX = oz_ex(SL, f - ke);
              oz_slice(Ls, f, ke, kb, ke, SL, EX);
              okf = oz_update(ring, gbar, fbar, afull, aempty, tmem, g, tcnt, &abort_s, SL, EX, f - ke, ke - kb, Ls, f,
                              w, W, r, ke, kE);
            }
          }
          // the rank-128 update of the rest of the front
          if (okf && kE < f) {
            int* EX = oz_ex(SL, f - kE);
            oz_slice(Ls, f, kE, kB, kE, SL, EX);
            okf = oz_update(ring, gbar, fbar, afull, aempty, tmem, g, tcnt, &abort_s, SL, EX, f - kE, kE - kB, Ls, f,
                            w, W, r, kE, f);
          }
        }
      }
      __syncthreads();
      if (P.sn_parent[gs] >= 0) {
        double* Uout = P.sn_hoff[gs] >= 0 ? hand + P.sn_hoff[gs] : stack + P.upd_ofs[gs];
        for (int64_t idx = tid; idx < (int64_t)r * r; idx += kThreads) Uout[idx] = W[idx];
      }
      __syncthreads();
    }
    if (tid == 0) {
      if (bad) atomicOr(status, kStatNotSPD);
      if (item.w >= 0 && !abort_s) {
        __threadfence();  // the task's factor panels and hand-over block before the count
        atomicAdd(tdone + item.w, 1);
      }
    }
    if (abort_s) break;
  }
  if (tid == 0 && abort_s) atomicOr(status, kStatTimeout);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// Smem of the solve (element type T of X).
template <typename T>
struct SolveSmem {
  T D[kNB][kNB + 1];
  T A[kNB][kT];
  T B[kNB][kT];  // also holds L_bb^{-1} (as [kNB][kNB + 1]) during the block solve
  T dinv[kNB];
};

// ---------------------------------------------------------------- tensor-core panel update of the TRSM
//
// C -= L_rs X_b for one 32-column block b of a supernode, on tcgen05: tiles
// of 128 rows (M) x 64 right-hand-side columns (N), K = the block's <= 32
// columns.  The CTA stages A (rows of L, FP64 -> FP32) and B (the solved rows
// of X) in the canonical 128-byte-swizzled K-major layout, one thread issues
// the MMAs into a 64-column TMEM accumulator and commits to an mbarrier, and
// the epilogue subtracts the accumulator (tcgen05.ld) from C.  MODE 1: TF32
// (kind::tf32); MODE 2: split-bf16, hi*hi + hi*lo + lo*hi (kind::f16).
constexpr int kTcRows = 128, kTcCols = 64;
constexpr uint32_t kTrsmTmemCols = 64;
constexpr int kTcMinRows = 128;  // smaller updates stay on the SIMT path (its per-tile set-up costs more there)
constexpr int kTcOpA = kTcRows * 128, kTcOpB = kTcCols * 128;

// Pipelined GEMM of the large fronts (gemm_tc): a ring of kGS stages, each holding one 32-deep K chunk of
// A (128 rows) and B (64 columns) as bf16 hi and lo halves in the 64-byte-swizzled K-major layout (rows of
// 64 bytes, 8-row atoms of 512 bytes), small enough that three CTAs stay resident per SM for the SIMT parts.
constexpr int kGS = 3;
constexpr int kGK = 32;                          // K values per chunk
constexpr int kGOpA = kTcRows * 64, kGOpB = kTcCols * 64;
constexpr int kGStage = 2 * kGOpA + 2 * kGOpB;  // 24 KB
constexpr int kTrsmDyn = 1024 + (kGS * kGStage > 2 * (kTcOpA + kTcOpB) ? kGS * kGStage : 2 * (kTcOpA + kTcOpB));

struct TcState {
  uint8_t* smem;     // 1024-aligned operand buffers: A (hi, lo), B (hi, lo); also the GEMM stage ring
  uint64_t* mbar;
  uint64_t* gbar;    // kGS stage barriers of the pipelined GEMM
  uint32_t tmem;
  uint32_t phase;    // commits so far (mbarrier parity)
  uint32_t g;        // GEMM chunks committed so far (stage = g % kGS, parity = (g / kGS) & 1)
  int* abort;        // shared flag: a bounded wait gave up
};

template <int MODE>
__device__ bool panel_update_tc(TcState& tc, const float* Ls, int f, int rbeg, int rend, int kbeg, int kend,
                                const float* Xs, int wp, float* Xw, float* W2, int w, int r, int J) {
  // C[rbeg .. rend) -= L[rbeg .. rend, kbeg .. kend) X[kbeg .. kend) (C = own rows of X below w, W2 beyond),
  // accumulated in TMEM over 32-deep chunks of K and written back once per 128 x 64 tile
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const uint32_t sA = smem_u32(tc.smem), sB = sA + (MODE == 2 ? 2 : 1) * kTcOpA;
  constexpr uint32_t idesc = idesc_m128(MODE == 2 ? 1u : 2u, (uint32_t)kTcCols);
  for (int ri = rbeg; ri < rend; ri += kTcRows) {
    for (int cj = 0; cj < J; cj += kTcCols) {
      for (int kc = kbeg; kc < kend; kc += kNB) {
        const int nk = min(kNB, kend - kc);
        // stage A: row m, 16-byte chunk c (K values 4c..4c+3 in TF32, 8c..8c+7 in bf16)
        for (int idx = tid; idx < kTcRows * 8; idx += kThreads) {
          const int m = idx % kTcRows, c = idx / kTcRows;
          const int i = ri + m;
          const uint32_t off = (m >> 3) * 1024 + (m & 7) * 128 + ((c ^ (m & 7)) << 4);
          if constexpr (MODE == 1) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int k = 4 * c + e;
              v[e] = (i < rend && k < nk) ? Ls[(int64_t)(kc + k) * f + i] : 0.f;
            }
            *reinterpret_cast<float4*>(tc.smem + off) = make_float4(v[0], v[1], v[2], v[3]);
          } else {
            __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int k = 8 * c + e;
              const float x = (i < rend && k < nk) ? Ls[(int64_t)(kc + k) * f + i] : 0.f;
              hi[e] = __float2bfloat16_rn(x);
              lo[e] = __float2bfloat16_rn(x - __bfloat162float(hi[e]));
            }
            *reinterpret_cast<uint4*>(tc.smem + off) = *reinterpret_cast<uint4*>(hi);
            *reinterpret_cast<uint4*>(tc.smem + kTcOpA + off) = *reinterpret_cast<uint4*>(lo);
          }
        }
        // stage B: right-hand-side column n, its solved K values kc .. kc + nk
        for (int idx = tid; idx < kTcCols * 8; idx += kThreads) {
          const int n = idx % kTcCols, c = idx / kTcCols;
          const int j = cj + n;
          const uint32_t off = (n >> 3) * 1024 + (n & 7) * 128 + ((c ^ (n & 7)) << 4);
          uint8_t* bB = tc.smem + (MODE == 2 ? 2 : 1) * kTcOpA;
          if constexpr (MODE == 1) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int k = 4 * c + e;
              v[e] = (j < J && k < nk) ? Xs[(int64_t)j * wp + kc + k] : 0.f;
            }
            *reinterpret_cast<float4*>(bB + off) = make_float4(v[0], v[1], v[2], v[3]);
          } else {
            __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int k = 8 * c + e;
              const float x = (j < J && k < nk) ? Xs[(int64_t)j * wp + kc + k] : 0.f;
              hi[e] = __float2bfloat16_rn(x);
              lo[e] = __float2bfloat16_rn(x - __bfloat162float(hi[e]));
            }
            *reinterpret_cast<uint4*>(bB + off) = *reinterpret_cast<uint4*>(hi);
            *reinterpret_cast<uint4*>(bB + kTcOpB + off) = *reinterpret_cast<uint4*>(lo);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t acc0 = kc > kbeg ? 1u : 0u;
          if constexpr (MODE == 1) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)  // K = 8 per MMA, 32 B of each 128-byte row
              mma_tf32(tc.tmem, sw128_desc(sA + kk * 32), sw128_desc(sB + kk * 32), idesc, (kk > 0) ? 1u : acc0);
          } else {
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {  // K = 16 per MMA; the chunk's 32 values fill half of each row
              const uint64_t ah = sw128_desc(sA + kk * 32), al = sw128_desc(sA + kTcOpA + kk * 32);
              const uint64_t bh = sw128_desc(sB + kk * 32), bl = sw128_desc(sB + kTcOpB + kk * 32);
              mma_f16(tc.tmem, ah, bh, idesc, (kk > 0) ? 1u : acc0);
              mma_f16(tc.tmem, ah, bl, idesc, 1u);
              mma_f16(tc.tmem, al, bh, idesc, 1u);
            }
          }
          mma_commit(smem_u32(tc.mbar));
          if (!mbar_wait(smem_u32(tc.mbar), tc.phase & 1)) *tc.abort = 1;
        }
        __syncthreads();
        tc.phase++;
        if (*tc.abort) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows), columns 32 (w / 4) .. + 31
      {
        const int q = warp % 4, ch = warp / 4;
        const int i = ri + q * 32 + lane;
        float* dst = i < w ? Xw + i : W2 + (i - w);
        const int64_t ld = i < w ? wp : r;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          uint32_t v[16];
          tmem_ld16(tc.tmem + ((uint32_t)(q * 32) << 16) + ch * 32 + h * 16, v);
          if (i < rend) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int j = cj + ch * 32 + h * 16 + e;
              if (j < J) dst[(int64_t)j * ld] -= __uint_as_float(v[e]);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
  }
  return true;
}

// SIMT update of the same form for smaller fronts: C[rbeg .. rend) -= L[., kbeg .. kend) X[kbeg .. kend),
// 64 x 64 register tiles accumulated over 32-deep chunks of K, written back once per tile.
template <typename T>
__device__ void panel_update_simt(SolveSmem<T>& sm, const T* Ls, int f, int rbeg, int rend, int kbeg, int kend,
                                  T* Xs, int wp, T* W2, int w, int r, int J) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16, warp = tid / 32;
  const int TR = (rend - rbeg + kT - 1) / kT, TC = (J + kT - 1) / kT;
  for (int ti = 0; ti < TR; ++ti) {
    for (int tcol = 0; tcol < TC; ++tcol) {
      const int ri = rbeg + ti * kT, cj = tcol * kT;
      // rows tx + 16u (all 16 tx per warp), columns ty + 16v (ty = 2 warp, 2 warp + 1)
      const int nu = groups16(rend - ri), nv = groups16(J - cj - 2 * warp);
      T acc[4][4] = {};
      for (int kc = kbeg; kc < kend; kc += kNB) {
        const int nk = min(kNB, kend - kc);
        for (int idx = tid; idx < kNB * kT; idx += kThreads) {
          int x = idx % kT, k = idx / kT;
          sm.A[k][x] = (k < nk && ri + x < rend) ? Ls[(int64_t)(kc + k) * f + ri + x] : (T)0;
        }
        for (int idx = tid; idx < kNB * kT; idx += kThreads) {
          int k = idx % kNB, y = idx / kNB;
          sm.B[k][y] = (k < nk && cj + y < J) ? Xs[(int64_t)(cj + y) * wp + kc + k] : (T)0;
        }
        __syncthreads();
        tile_mma_dispatch<T, false>(sm.A, sm.B, nk, acc, tx, ty, nu, nv);
        __syncthreads();
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        int col = cj + ty + 16 * v;
        if (v >= nv || col >= J) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          int i = ri + tx + 16 * u;
          if (u >= nu || i >= rend) continue;
          if (i < w) Xs[(int64_t)col * wp + i] -= acc[u][v];
          else W2[(int64_t)col * r + (i - w)] -= acc[u][v];
        }
      }
    }
  }
}

// C[rbeg, rend) x [0, J) -= A[rbeg, rend) x [kbeg, kend) . B[kbeg, kend) x [0, J) on the tensor cores in split
// bf16 (hi*hi + hi*lo + lo*hi, FP32 accumulation in TMEM), for the large fronts.  A is the row-major hi/lo copy
// of the supernode's panel (row i: lwp hi values, then lwp lo values; zero beyond w), B the bf16 hi/lo copy of
// X_s (column j: wp hi values, then wp lo values; zero beyond w).  kbeg is a multiple of 8 and every K value
// in [kbeg, kend) rounded up to 8 lies inside the padding.  Tiles of 128 rows x 64 columns, K in chunks of 32
// (one swizzled 64-byte row per operand row): all threads stage chunks by cp.async into the kGS-stage ring,
// running ahead across tile boundaries, one thread issues each chunk's MMAs and commits them to its stage's
// mbarrier (which frees the stage), and after a tile's last chunk the CTA subtracts the accumulator from C
// (rows below w: the own rows of X_s; the others: W2, or with W2out, W2out = W2 - accumulator, the parent's
// update block written in place).  Every wait is bounded.
__device__ bool gemm_tc(TcState& tc, const uint16_t* LH, int lwp, int rbeg, int rend, int kbeg, int kend,
                        const uint16_t* X2s, int wp, float* Xs, float* W2, int w, int r, int J,
                        float* W2out = nullptr) {
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int ntm = (rend - rbeg + kTcRows - 1) / kTcRows, ntn = (J + kTcCols - 1) / kTcCols;
  const int nck = (kend - kbeg + kGK - 1) / kGK;
  const int total = ntm * ntn * nck;
  if (rend <= rbeg || J <= 0 || kend <= kbeg) return true;
  const uint32_t sb0 = smem_u32(tc.smem);
  const uint32_t g0 = tc.g;
  constexpr uint32_t idesc = idesc_m128(1u, (uint32_t)kTcCols);
  auto load = [&](int q, uint32_t sbase) {
    const int ck = q % nck, t = q / nck, tn = t % ntn, tm = t / ntn;
    const int k0 = kbeg + ck * kGK, i0 = rbeg + tm * kTcRows, j0 = tn * kTcCols;
    // 4 pieces of 16 B (8 bf16) per 64-byte row
    for (int idx = tid; idx < 2 * kTcRows * 4 + 2 * kTcCols * 4; idx += kThreads) {
      uint32_t dst;
      const void* src;
      bool ok;
      if (idx < 2 * kTcRows * 4) {
        const int part = idx / (kTcRows * 4), rem = idx % (kTcRows * 4), m = rem / 4, c = rem % 4;
        const int i = i0 + m, k = k0 + 8 * c;
        ok = i < rend && k < kend;
        src = ok ? (const void*)(LH + (int64_t)i * 2 * lwp + (part ? lwp : 0) + k) : (const void*)LH;
        dst = sbase + part * kGOpA + (m >> 3) * 512 + (m & 7) * 64 + ((c ^ ((m >> 1) & 3)) << 4);
      } else {
        const int id2 = idx - 2 * kTcRows * 4;
        const int part = id2 / (kTcCols * 4), rem = id2 % (kTcCols * 4), n = rem / 4, c = rem % 4;
        const int j = j0 + n, k = k0 + 8 * c;
        ok = j < J && k < kend;
        src = ok ? (const void*)(X2s + (int64_t)j * 2 * wp + (part ? wp : 0) + k) : (const void*)X2s;
        dst = sbase + 2 * kGOpA + part * kGOpB + (n >> 3) * 512 + (n & 7) * 64 + ((c ^ ((n >> 1) & 3)) << 4);
      }
      cp_async16(dst, src, ok);
    }
  };
  bool ok = true;
  for (int i = 0; i < total + kGS - 1; ++i) {
    if (i < total) {
      if (i >= kGS) {  // the stage's previous chunk must have been multiplied
        const uint32_t gp = g0 + i - kGS;
        if (tid == 0 && !mbar_wait(smem_u32(&tc.gbar[gp % kGS]), (gp / kGS) & 1)) *tc.abort = 1;
        __syncthreads();
        if (*tc.abort) {
          ok = false;
          break;
        }
      }
      load(i, sb0 + ((g0 + i) % kGS) * kGStage);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    const int j = i - (kGS - 1);
    if (j < 0 || j >= total) continue;
    asm volatile("cp.async.wait_group %0;" ::"n"(kGS - 1) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const int ck = j % nck;
    const uint32_t st = (g0 + j) % kGS;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sA = sb0 + st * kGStage, sB = sA + 2 * kGOpA;
#pragma unroll
      for (int kk = 0; kk < kGK / 16; ++kk) {  // K = 16 per MMA, 32 B of each 64-byte row
        const uint64_t ah = sw64_desc(sA + kk * 32), al = sw64_desc(sA + kGOpA + kk * 32);
        const uint64_t bh = sw64_desc(sB + kk * 32), bl = sw64_desc(sB + kGOpB + kk * 32);
        mma_f16(tc.tmem, ah, bh, idesc, (ck > 0 || kk > 0) ? 1u : 0u);
        mma_f16(tc.tmem, ah, bl, idesc, 1u);
        mma_f16(tc.tmem, al, bh, idesc, 1u);
      }
      mma_commit(smem_u32(&tc.gbar[st]));
    }
    if (ck != nck - 1) continue;
    // the tile's last chunk: wait for its MMAs, then C -= accumulator
    if (tid == 0 && !mbar_wait(smem_u32(&tc.gbar[st]), ((g0 + j) / kGS) & 1)) *tc.abort = 1;
    __syncthreads();
    if (*tc.abort) {
      ok = false;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    {
      const int t = j / nck, tn = t % ntn, tm = t / ntn;
      const int ri = rbeg + tm * kTcRows, cj = tn * kTcCols;
      const int q = warp % 4, ch = warp / 4;
      const int row = ri + q * 32 + lane;
      const float* src = row < w ? Xs + row : W2 + (row - w);
      float* dst = row < w ? Xs + row : (W2out ? W2out : W2) + (row - w);
      const int64_t ld = row < w ? wp : r;
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {  // 16 columns per TMEM load (fewer live registers)
        uint32_t v[16];
        tmem_ld16(tc.tmem + ((uint32_t)(q * 32) << 16) + ch * 32 + h * 16, v);
        if (row < rend) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int col = cj + ch * 32 + h * 16 + e;
            if (col < J) dst[(int64_t)col * ld] = src[(int64_t)col * ld] - __uint_as_float(v[e]);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (!ok) asm volatile("cp.async.wait_all;" ::: "memory");
  tc.g = g0 + total;
  return ok;
}

// Write the bf16 hi/lo copy of rows [ka, kb) of X_s (column j: wp hi values, then wp lo values).
__device__ __forceinline__ void write_x2(const float* Xs, int wp, uint16_t* X2s, int ka, int kb, int J) {
  const int nk = kb - ka;
  __nv_bfloat16* h2 = reinterpret_cast<__nv_bfloat16*>(X2s);
  for (int64_t idx = threadIdx.x; idx < (int64_t)nk * J; idx += kThreads) {
    const int64_t j = idx / nk;
    const int k = ka + (int)(idx - j * nk);
    const float v = Xs[j * wp + k];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    h2[2 * j * wp + k] = hi;
    h2[2 * j * wp + wp + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

// Diagonal step of the forward solve: X_b <- L_bb^{-1} X_b for the rows [kb, kb + nbk) of X_s (all J columns),
// with L_bb^{-1} formed explicitly by one warp (a 32 x 32 triangular inverse) and applied as a small GEMM.
template <typename T>
__device__ void diag_block(SolveSmem<T>& sm, const T* Ls, int f, int kb, int nbk, T* Xs, int wp, int J, int unit) {
  const int tid = threadIdx.x, warp = tid / 32;
  auto Di = reinterpret_cast<T (*)[kNB + 1]>(&sm.B[0][0]);
  for (int idx = tid; idx < kNB * kNB; idx += kThreads) {
    int i = idx % kNB, j = idx / kNB;
    sm.D[i][j] = (i < nbk && j <= i) ? Ls[(int64_t)(kb + j) * f + kb + i] : (T)0;
  }
  // unit: L is in unit-lower form (pivots folded out after the assembly), its stored diagonal is zero
  if (tid < kNB) sm.dinv[tid] = tid < nbk ? (unit ? (T)1 : (T)1 / Ls[(int64_t)(kb + tid) * f + kb + tid]) : (T)0;
  __syncthreads();
  if (warp == 0) warp_tri_inverse<T>(sm.D, sm.dinv, Di, nbk);
  __syncthreads();
  // X_b <- Di X_b for 64 columns at a time: column y = tid % 64, rows jg*8 .. jg*8+7
  const int y = tid % kT, jg = tid / kT;
  for (int cj = 0; cj < J; cj += kT) {
    for (int idx = tid; idx < kNB * kT; idx += kThreads) {
      int k = idx % kNB, yy = idx / kNB;
      sm.A[k][yy] = (k < nbk && cj + yy < J) ? Xs[(int64_t)(cj + yy) * wp + kb + k] : (T)0;
    }
    __syncthreads();
    if (jg * 8 < nbk && cj + (y & ~31) < J) {
      T acc[8] = {};
      for (int k = 0; k <= min(nbk - 1, jg * 8 + 7); ++k) {
        const T a = sm.A[k][y];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[jj] = fma(Di[jg * 8 + jj][k], a, acc[jj]);
      }
      if (cj + y < J) {
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int j = jg * 8 + jj;
          if (j < nbk) Xs[(int64_t)(cj + y) * wp + kb + j] = acc[jj];
        }
      }
    }
    __syncthreads();
  }
}

// Forward solve of one RHS front: X_s = L_ss^{-1} X_s, then C -= L_rs X_s
// (C = the r bottom rows).  Column-major fronts: column j of X_s is
// Xs[j * wp + 0 .. w), column j of the bottom block is W2[j * r + 0 .. r).
// L is read in the solve's precision T (the mixed path reads the FP32 copy of
// L).  The own rows are solved right-looking in 32-row blocks: each block is
// applied as its explicit inverse (a small GEMM), then the own rows below it
// are updated.  The bottom rows are updated once at the end with K = w
// (accumulated over all blocks before one write-back of W2).
template <typename T>
__device__ bool solve_front(SolveSmem<T>& sm, const T* Ls, int f, int w, T* Xs, int wp, T* W2, int J,
                            TcState* tc, int tcmode, int unit) {
  const int r = f - w;
  for (int kb = 0; kb < w; kb += kNB) {
    const int nbk = min(kNB, w - kb);
    diag_block<T>(sm, Ls, f, kb, nbk, Xs, wp, J, unit);
    // the own rows below the block
    const int i0 = kb + nbk;
    if (i0 < w) {
      if constexpr (sizeof(T) == 4) {
        if (tcmode > 0 && w - i0 >= kTcMinRows) {
          const bool ok = tcmode == 1 ? panel_update_tc<1>(*tc, Ls, f, i0, w, kb, i0, Xs, wp, Xs, W2, w, r, J)
                                      : panel_update_tc<2>(*tc, Ls, f, i0, w, kb, i0, Xs, wp, Xs, W2, w, r, J);
          if (!ok) return false;
          continue;
        }
      }
      panel_update_simt<T>(sm, Ls, f, i0, w, kb, i0, Xs, wp, W2, w, r, J);
    }
  }
  // the bottom rows: W2 -= L_rs X_s, K = w
  if (r > 0) {
    if constexpr (sizeof(T) == 4) {
      if (tcmode > 0 && r >= kTcMinRows) {
        const bool ok = tcmode == 1 ? panel_update_tc<1>(*tc, Ls, f, w, f, 0, w, Xs, wp, Xs, W2, w, r, J)
                                    : panel_update_tc<2>(*tc, Ls, f, w, f, 0, w, Xs, wp, Xs, W2, w, r, J);
        return ok;
      }
    }
    panel_update_simt<T>(sm, Ls, f, w, f, 0, w, Xs, wp, W2, w, r, J);
  }
  return true;
}

// Shared memory of the 128-row diagonal solve of a large front (aliases the GEMM ring, which is idle then).
struct Diag128Smem {
  float Di[4][kNB][kNB + 1];  // inverses of the four 32 x 32 diagonal blocks
  float Lo[6][kNB][kNB + 1];  // the six 32 x 32 blocks below the diagonal: (1,0) (2,0) (2,1) (3,0) (3,1) (3,2)
  float Xb[kTcRows][kNB + 1]; // 32 right-hand-side columns of the block's rows
};
static_assert(sizeof(Diag128Smem) <= kGS * kGStage, "the diagonal solve fits in the GEMM ring");

__device__ __forceinline__ int lo_pair(int a, int b) { return a == 1 ? 0 : a == 2 ? 1 + b : 3 + b; }  // a > b

// X_b <- L_bb^{-1} X_b for the rows [k0, k0 + nr) (nr <= 128) of X_s, all J columns, in shared memory: with the
// inverses of the four 32 x 32 diagonal blocks of L_bb (Dinv, from l16_kernel), 32 columns at a time the block
// rows are loaded, solved by sub-block (the sub-block's inverse applied, then the sub-blocks below it updated
// with the blocks of L_bb below the diagonal) and written back together with their bf16 hi/lo copy (with the
// zero padding rows [w, wp) after the last block).  keep_x = false: the solved rows go to the hi/lo copy only
// (nothing reads their FP32 values afterwards when the SYRK takes the hi/lo copy).
__device__ void diag128(Diag128Smem& d, const float* Ls, const float* Dinv, int f, int w, int k0, int nr, float* Xs,
                        int wp, int J, uint16_t* X2s, bool keep_x) {
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int nsb = (nr + kNB - 1) / kNB;
  // the inverted diagonal blocks (l16_kernel) and the L blocks below the diagonal (FP32 copy of L, column-major
  // f x w panel)
  for (int idx = tid; idx < nsb * kNB * kNB; idx += kThreads) {
    const int b = idx / (kNB * kNB), rem = idx % (kNB * kNB);
    d.Di[b][rem / kNB][rem % kNB] = Dinv[idx];
  }
  for (int idx = tid; idx < 6 * kNB * kNB; idx += kThreads) {
    const int q = idx / (kNB * kNB), rem = idx % (kNB * kNB), i = rem % kNB, j = rem / kNB;
    const int a = q == 0 ? 1 : q <= 2 ? 2 : 3, b = q == 0 ? 0 : q <= 2 ? q - 1 : q - 3;  // block row, column
    const int gi = a * kNB + i, gj = b * kNB + j;
    d.Lo[q][i][j] = (a < nsb && gi < nr) ? Ls[(int64_t)(k0 + gj) * f + k0 + gi] : 0.f;
  }
  __syncthreads();
  const int rowsp = (k0 + nr == w) ? wp - k0 : nr;  // rows written to X2 (the padding after the last block)
  __nv_bfloat16* h2 = reinterpret_cast<__nv_bfloat16*>(X2s);
  for (int cj = 0; cj < J; cj += kNB) {
    for (int idx = tid; idx < kTcRows * kNB; idx += kThreads) {
      const int i = idx % kTcRows, y = idx / kTcRows;
      d.Xb[i][y] = (i < nr && cj + y < J) ? Xs[(int64_t)(cj + y) * wp + k0 + i] : 0.f;
    }
    __syncthreads();
    for (int sb = 0; sb < nsb; ++sb) {
      // X_sb <- Di_sb X_sb: lane = column, rows 4 warp .. 4 warp + 3 of the sub-block
      float acc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = 4 * warp + u;
        float a = 0.f;
        for (int k = 0; k <= i; ++k) a = fmaf(d.Di[sb][i][k], d.Xb[sb * kNB + k][lane], a);
        acc[u] = a;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 4; ++u) d.Xb[sb * kNB + 4 * warp + u][lane] = acc[u];
      __syncthreads();
      // the sub-blocks below: X_a -= L_(a,sb) X_sb
      for (int a = sb + 1; a < nsb; ++a) {
        const int pq = lo_pair(a, sb);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = 4 * warp + u;
          float s = 0.f;
#pragma unroll 8
          for (int k = 0; k < kNB; ++k) s = fmaf(d.Lo[pq][i][k], d.Xb[sb * kNB + k][lane], s);
          d.Xb[a * kNB + i][lane] -= s;
        }
      }
      __syncthreads();
    }
    // write back X and its bf16 hi/lo copy
    for (int idx = tid; idx < kTcRows * kNB; idx += kThreads) {
      const int i = idx % kTcRows, y = idx / kTcRows;
      if (cj + y < J && i < rowsp) {
        const float v = i < nr ? d.Xb[i][y] : 0.f;
        if (keep_x && i < nr) Xs[(int64_t)(cj + y) * wp + k0 + i] = v;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const int64_t o = 2 * (int64_t)(cj + y) * wp + k0 + i;
        h2[o] = hi;
        h2[o + wp] = __float2bfloat16_rn(v - __bfloat162float(hi));
      }
    }
    __syncthreads();
  }
}

// Forward solve of a large front on the tensor cores (mixed precision): the own rows in blocks of 128, each
// solved by four diagonal steps of 32 rows (the rows inside the block updated on the SIMT path), its rows
// written as bf16 hi/lo (the B operand of the later GEMMs and of the split-bf16 SYRK), then the own rows below
// it updated with K = 128 by the pipelined GEMM; finally the bottom rows, W2 -= L_rs X_s with K = w, by the same
// GEMM.  LH: the row-major hi/lo copy of the panel (launch_l16).  X2s: the hi/lo copy of X_s.
__device__ bool solve_front_big(SolveSmem<float>& sm, const float* Ls, const uint16_t* LH, const float* Dinv, int f,
                                int w, float* Xs, int wp, float* W2, int J, uint16_t* X2s, TcState& tc, bool keep_x,
                                float* Uout) {
  const int r = f - w;
  Diag128Smem& d = *reinterpret_cast<Diag128Smem*>(tc.smem);
  for (int k0 = 0; k0 < w; k0 += kTcRows) {
    const int e0 = min(w, k0 + kTcRows);
    diag128(d, Ls, Dinv + (int64_t)(k0 / kNB) * kNB * kNB, f, w, k0, e0 - k0, Xs, wp, J, X2s, keep_x);
    if (e0 < w && !gemm_tc(tc, LH, wp, e0, w, k0, e0, X2s, wp, Xs, W2, w, r, J)) return false;
  }
  if (r > 0 && !gemm_tc(tc, LH, wp, w, f, 0, w, X2s, wp, Xs, W2, w, r, J, Uout)) return false;
  return true;
}

// Round an FP32 value to TF32 (10 explicit mantissa bits), to nearest with ties away from zero.
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// tcmode (FP32 X only): 0 = SIMT panel updates, 1 = TF32 tensor cores, 2 = split-bf16 tensor cores.
// tf32_out (FP32 X only): round each finished X block to TF32, so that the TF32 SYRK that reads it
// multiplies operands rounded to nearest (the tensor cores would otherwise drop the low 13 bits).
// unit (FP64 X only): solve with the unit-lower L_u that the assembly leaves (X_u = L_u^{-1} P B^T).
// Work items (subdomain, first sorted column ca) cover the columns [ca, ca + cw) (cw = 0: all of them):
// the columns of X are independent, so a subdomain's columns can be split over several CTAs.  Every
// supernode then handles J_s restricted to the block; the restricted ranges nest like J_s itself.
// X2 (FP32 X only): also write each finished block as bf16 hi/lo halves (hi = bf16(x), lo = bf16(x - hi)),
// per column wp hi values then wp lo values, for the split-bf16 SYRK.
// LT: the factor in the solve's precision (the FP32 copy of L for T = float, L itself for T = double).
template <typename T>
__global__ void __launch_bounds__(kThreads, 3)
    trsm_kernel(DevPlan P, const int2* items, int nitems, int cw, int* queue, const T* LT, T* X, T* ws,
                int64_t ws_stride, int64_t front_sz, int tcmode, int tf32_out, int unit, uint16_t* X2, int x2_out,
                int* status) {
  __shared__ uint64_t tc_mbar;
  __shared__ uint64_t tc_gbar[kGS];
  __shared__ uint32_t tc_tmem;
  __shared__ int tc_abort;
  extern __shared__ uint8_t tc_raw[];
  // the SIMT solve's buffers share the dynamic shared memory with the tensor-core operand buffers (never in
  // use at the same time)
  // (the offset is added to the shared array itself, so the compiler keeps shared-memory loads and stores)
  uint8_t* dyn = tc_raw + ((1024u - (smem_u32(tc_raw) & 1023u)) & 1023u);
  SolveSmem<T>& sm = *reinterpret_cast<SolveSmem<T>*>(dyn);
  const int tid = threadIdx.x;
  T* W2 = ws + (int64_t)blockIdx.x * ws_stride;
  T* stack = W2 + front_sz;
  TcState tc{};
  // the tcgen05 code exists only in the FP32 instantiation: with it compiled into the FP64 one (and skipped
  // at run time) the FP64 TRSM took 24.7 instead of 15.0 ms on the 1024-subdomain 2D workload
  if constexpr (sizeof(T) != 4) tcmode = 0;
  if constexpr (sizeof(T) == 4) {
  if (tcmode > 0) {
    if (tid < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tc_tmem)),
                   "r"(kTrsmTmemCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tc_mbar)));
      for (int k = 0; k < kGS; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tc_gbar[k])));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      tc_abort = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tc.smem = dyn;
    tc.mbar = &tc_mbar;
    tc.gbar = tc_gbar;
    tc.tmem = tc_tmem;
    tc.phase = 0;
    tc.g = 0;
    tc.abort = &tc_abort;
  }
  }
  for (;;) {
    int it = pop_item(queue);
    if (it >= nitems) break;
    const int si = items[it].x;
    const int ca = items[it].y, cb = cw > 0 ? ca + cw : 0x7fffffff;
    const SubInfo S = P.sub[si];
    const T* L = LT + S.L;
    T* Xsub = X + S.X;
    for (int a = 0; a < S.nact; ++a) {
      const int s = P.act[S.act0 + a];
      const int gs = S.sn0 + s, bs = S.bsn0 + s;
      const int c0 = P.sn_c0[gs], w = P.sn_w[gs], r = P.sn_r[gs], f = w + r;
      const int wp = (w + 7) & ~7;
      const int jb = max(P.jb[bs], ca), je = min(P.je[bs], cb), jo = max(P.jo[bs], ca);
      const int J = je - jb;
      if (J <= 0) continue;  // no column of this block reaches s (nor any of its descendants)
      T* Xs = Xsub + P.Xofs[bs] + (int64_t)(jb - P.jb[bs]) * wp;
      for (int64_t idx = tid; idx < (int64_t)wp * J; idx += kThreads) Xs[idx] = (T)0;
      for (int64_t idx = tid; idx < (int64_t)r * J; idx += kThreads) W2[idx] = (T)0;
      __syncthreads();
      for (int j = jo + tid; j < je; j += kThreads) {
        int row = P.spos[S.col0 + j] - c0;
        Xs[(int64_t)(j - jb) * wp + row] = (T)P.qsign[S.qcol + j];
      }
      for (int c = P.ch_off[gs]; c < P.ch_off[gs + 1]; ++c) {
        const int lc = P.ch_list[c];
        const int gc = S.sn0 + lc, bc = S.bsn0 + lc;
        const int jbc = max(P.jb[bc], ca), Jc = min(P.je[bc], cb) - jbc;
        if (Jc <= 0) continue;
        const int rc = P.sn_r[gc], coff = jbc - jb;
        const T* U = stack + P.rhs_ofs[bc];
        const int* rl = P.rel + P.rel_off[gc];
        // children own disjoint column ranges: no conflicts between them.  Four elements per thread and step,
        // their loads issued before their read-modify-writes (the targets are distinct: rel is one-to-one)
        const int64_t n = (int64_t)rc * Jc;
        for (int64_t base = tid; base < n; base += 4 * kThreads) {
          T* dst[4];
          T v[4], cur[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int64_t idx = base + (int64_t)u * kThreads;
            dst[u] = nullptr;
            if (idx < n) {
              const int col = (int)(idx / rc), a2 = (int)(idx - (int64_t)col * rc);
              const int ra = rl[a2];
              v[u] = U[idx];
              dst[u] = ra < w ? Xs + (int64_t)(coff + col) * wp + ra : W2 + (int64_t)(coff + col) * r + (ra - w);
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) cur[u] = dst[u] ? *dst[u] : (T)0;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (dst[u]) *dst[u] = cur[u] + v[u];
        }
      }
      __syncthreads();
      // large fronts of the tensor-core path: the blocked solve with pipelined GEMMs
      const int64_t lho = (sizeof(T) == 4 && tcmode == 2) ? P.lh_ofs[gs] : -1;
      uint16_t* X2s = X2 ? X2 + 2 * (S.X + P.Xofs[bs] + (int64_t)(jb - P.jb[bs]) * wp) : nullptr;
      bool ok;
      if constexpr (sizeof(T) == 4) {
        // the parent's update block is written by the bottom GEMM's epilogue (after the children's blocks on the
        // stack, which it may overwrite, have been read)
        ok = lho >= 0 && X2s ? solve_front_big(sm, L + P.Lofs[gs], P.LH + S.lh + lho, P.DI + S.di + P.di_ofs[gs], f,
                                               w, Xs, wp, W2, J, X2s, tc, !x2_out,
                                               P.sn_parent[gs] >= 0 ? stack + P.rhs_ofs[bs] : nullptr)
                             : solve_front<T>(sm, L + P.Lofs[gs], f, w, Xs, wp, W2, J, &tc, tcmode, unit);
      } else {
        ok = solve_front<T>(sm, L + P.Lofs[gs], f, w, Xs, wp, W2, J, &tc, tcmode, unit);
      }
      if (!ok) break;
      __syncthreads();
      if constexpr (sizeof(T) == 4) {
        // X_s is final here (the parent reads only the bottom rows W2)
        if (tf32_out)
          for (int64_t idx = tid; idx < (int64_t)wp * J; idx += kThreads) Xs[idx] = round_tf32(Xs[idx]);
        if (X2 && x2_out && !(lho >= 0)) {
          __nv_bfloat16* h2 =
              reinterpret_cast<__nv_bfloat16*>(X2) + 2 * (S.X + P.Xofs[bs] + (int64_t)(jb - P.jb[bs]) * wp);
          for (int64_t idx = tid; idx < (int64_t)wp * J; idx += kThreads) {
            const int64_t j = idx / wp, k = idx - j * wp;
            const float v = Xs[idx];
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            h2[2 * j * wp + k] = hi;
            h2[2 * j * wp + wp + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
          }
        }
      }
      if (P.sn_parent[gs] >= 0 && !(lho >= 0 && X2s && r > 0)) {
        T* dst = stack + P.rhs_ofs[bs];
        for (int64_t idx = tid; idx < (int64_t)r * J; idx += kThreads) dst[idx] = W2[idx];
      }
      __syncthreads();
    }
    if (tcmode > 0 && tc_abort) break;
  }
  if constexpr (sizeof(T) == 4) {
  if (tcmode > 0) {
    // a timed-out wait leaves the MMA unconfirmed: report it; TMEM is released either way
    if (tid == 0 && tc_abort) atomicOr(status, kStatTimeout);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid < 32) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc.tmem), "r"(kTrsmTmemCols));
    }
  }
  }
}

// FP32 copy of the factor for the mixed-precision TRSM (one conversion per entry instead of one per use;
// FP64 -> FP32 conversions run on the narrow FP64 pipe of this GPU)
__global__ void __launch_bounds__(256) l32_kernel(const double* __restrict__ L, float* __restrict__ L32, int64_t n) {
  const int64_t n2 = n / 2;
  const double2* L2 = reinterpret_cast<const double2*>(L);
  float2* O2 = reinterpret_cast<float2*>(L32);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = L2[i];
    O2[i] = make_float2((float)v.x, (float)v.y);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) L32[n - 1] = (float)L[n - 1];
}

// Row-major bf16 hi/lo copy of the large panels for the tensor-core TRSM: row i of the f x w panel as lwp hi
// values then lwp lo values (hi = bf16(x), lo = bf16(x - hi) of the FP32 entry, zero for k >= w), so that
// every 16-byte piece of a K-major operand row is one cp.async.  Each warp transposes 32 x 32 tiles of a
// panel on its own (no CTA-wide barrier: the eight warps of a CTA keep eight tiles in flight).  Also the
// inverses of the panel's 32 x 32 diagonal blocks (FP32, one warp per block, from the same FP32 entries), which
// every column block of the TRSM then reads instead of recomputing them.
__global__ void __launch_bounds__(256) l16_kernel(DevPlan P, const int2* items, int nitems, const float* L32,
                                                  uint16_t* LH, float* DI) {
  __shared__ float t[8][32][33];
  __shared__ float dv[4][kNB];
  const int lane = threadIdx.x % 32, wq = threadIdx.x / 32;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const SubInfo S = P.sub[items[it].x];
    const int gs = S.sn0 + items[it].y;
    const int w = P.sn_w[gs], f = w + P.sn_r[gs], lwp = (w + 7) & ~7;
    const float* Lp = L32 + S.L + P.Lofs[gs];
    __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(LH + S.lh + P.lh_ofs[gs]);
    const int nti = (f + 31) / 32, ntk = (lwp + 31) / 32;
    for (int q = wq; q < nti * ntk; q += 8) {
      const int i0 = (q / ntk) * 32, k0 = (q % ntk) * 32;
      // lane = row: column k of the tile is 32 consecutive rows of the column-major panel
#pragma unroll 8
      for (int kk = 0; kk < 32; ++kk) {
        const int k = k0 + kk, i = i0 + lane;
        t[wq][kk][lane] = (i < f && k < w) ? Lp[(int64_t)k * f + i] : 0.f;
      }
      __syncwarp();
      // lane = column: row i of the tile is 32 consecutive entries of the row-major copy
      for (int ii = 0; ii < 32; ++ii) {
        const int i = i0 + ii, k = k0 + lane;
        if (i < f && k < lwp) {
          const float v = t[wq][lane][ii];
          const __nv_bfloat16 hi = __float2bfloat16_rn(v);
          out[(int64_t)i * 2 * lwp + k] = hi;
          out[(int64_t)i * 2 * lwp + lwp + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
        }
      }
      __syncwarp();
    }
    // the diagonal blocks: warps 0-3 invert blocks wq, wq + 4, ... (the L block in t[wq], its inverse in
    // t[wq + 4], free once every warp has finished its tiles); block b covers own rows 32 b .. 32 b + 31, 4 blocks
    // per 128 rows, the slots of blocks past w stay unwritten and unread
    __syncthreads();
    float* di = DI + S.di + P.di_ofs[gs];
    for (int b = wq; wq < 4 && b < (w + kNB - 1) / kNB; b += 4) {
      const int nbk = min(kNB, w - b * kNB);
      for (int j = 0; j < kNB; ++j)  // lane = row, one column at a time (coalesced)
        t[wq][lane][j] = (lane < nbk && j <= lane) ? Lp[(int64_t)(b * kNB + j) * f + b * kNB + lane] : 0.f;
      dv[wq][lane] = lane < nbk ? 1.f / Lp[(int64_t)(b * kNB + lane) * f + b * kNB + lane] : 0.f;
      __syncwarp();
      warp_tri_inverse<float>(reinterpret_cast<const float (*)[kNB + 1]>(&t[wq][0][0]), dv[wq],
                              reinterpret_cast<float (*)[kNB + 1]>(&t[wq + 4][0][0]), nbk);
      for (int i = 0; i < kNB; ++i) di[(int64_t)b * kNB * kNB + i * kNB + lane] = t[wq + 4][i][lane];
      __syncwarp();
    }
    __syncthreads();  // t is free again for the next panel's tiles
  }
}

}  // namespace

void launch_l16(const DevPlan& P, const int2* items, int nitems, const float* L32, uint16_t* LH, float* DI, int grid,
                cudaStream_t st) {
  if (nitems > 0) l16_kernel<<<std::min(grid, nitems), 256, 0, st>>>(P, items, nitems, L32, LH, DI);
}

void launch_l32(const double* L, float* L32, int64_t n, int grid, cudaStream_t st) {
  if (n > 0) l32_kernel<<<grid, 256, 0, st>>>(L, L32, n);
}

void launch_chol(const DevPlan& P, const int4* items, int nitems, int use_tasks, int* queue, int* tdone,
                 double* hand, double* ws, int64_t ws_stride, int64_t front_sz, int64_t stack_sz, int grid,
                 int* status, cudaStream_t st, int flags) {
  const int smem = kFrontSmem * 8;
  cudaFuncSetAttribute(chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  chol_kernel<<<grid, kThreads, smem, st>>>(P, items, nitems, use_tasks, queue, tdone, hand, ws, ws_stride, front_sz,
                                            stack_sz, flags, status);
}

void launch_chol_tc(const DevPlan& P, const int4* items, int nitems, int* queue, int* tdone, double* hand,
                    double* ws, int64_t ws_stride, int64_t front_sz, uint16_t* slices, int64_t slice_stride, int grid,
                    int* status, cudaStream_t st, int flags) {
  if (nitems <= 0) return;
  cudaFuncSetAttribute(chol_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCholTcDyn);
  chol_tc_kernel<<<std::min(grid, nitems), kThreads, kCholTcDyn, st>>>(P, items, nitems, queue, tdone, hand, ws,
                                                                       ws_stride, front_sz, slices, slice_stride,
                                                                       flags, status);
}

int64_t chol_tc_scratch(int fmax) {
  const int64_t npad = (fmax + kOzM - 1) / kOzM * kOzM;
  return (npad * (2 * kOzS * kOzK + 2) + 127) / 128 * 128;
}

int chol_ctas_per_sm() {
  const int smem = kFrontSmem * 8;
  cudaFuncSetAttribute(chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, chol_kernel, kThreads, smem);
  return nb > 0 ? nb : 1;
}

static int trsm_smem(bool fp32, int tcmode) {
  if (!fp32) return 1024 + (int)sizeof(SolveSmem<double>);
  return tcmode > 0 ? kTrsmDyn : 1024 + (int)sizeof(SolveSmem<float>);
}

void launch_trsm(const DevPlan& P, const int2* items, int nitems, int cw, int* queue, void* X, bool fp32,
                 double* ws, int64_t ws_stride, int64_t front_sz, int grid, int tcmode, int tf32_out, int* status,
                 cudaStream_t st, int unit, uint16_t* X2, const float* L32, int x2_out) {
  const int smem = trsm_smem(fp32, tcmode);
  if (fp32) {
    cudaFuncSetAttribute(trsm_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(trsm_kernel<float>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    trsm_kernel<float><<<grid, kThreads, smem, st>>>(P, items, nitems, cw, queue, L32, (float*)X, (float*)ws,
                                                     2 * ws_stride, front_sz, tcmode, tf32_out, 0, X2, x2_out,
                                                     status);
  } else {
    cudaFuncSetAttribute(trsm_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    trsm_kernel<double><<<grid, kThreads, smem, st>>>(P, items, nitems, cw, queue, P.L, (double*)X, ws, ws_stride,
                                                      front_sz, 0, 0, unit, nullptr, 0, status);
  }
}

// Resident CTAs per SM of the TRSM, from its registers and shared memory.  (The occupancy API answers 1 for
// the FP32 kernel, which allocates tensor memory, although three of its CTAs run side by side: 3 x 64 TMEM
// columns fit the SM's 512.  The TRSM's CTAs never wait on one another, so a grid above what fits is only
// scheduled later, never blocked.)
int trsm_ctas_per_sm(bool fp32, int tcmode) {
  const int smem = trsm_smem(fp32, tcmode);
  cudaFuncAttributes fa{};
  if (fp32) {
    cudaFuncSetAttribute(trsm_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(trsm_kernel<float>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    if (cudaFuncGetAttributes(&fa, trsm_kernel<float>) != cudaSuccess) return 1;
  } else {
    cudaFuncSetAttribute(trsm_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (cudaFuncGetAttributes(&fa, trsm_kernel<double>) != cudaSuccess) return 1;
  }
  int dev = 0, sm_smem = 0, reserved = 0, sm_regs = 0, sm_threads = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&sm_threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  const int per_cta_smem = smem + (int)fa.sharedSizeBytes + reserved;
  const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;  // allocated per warp in units of 256
  int nb = std::min(sm_smem / std::max(per_cta_smem, 1), sm_regs / std::max(regs_warp * (kThreads / 32), 1));
  nb = std::min(nb, sm_threads / kThreads);
  if (fp32 && tcmode > 0) nb = std::min(nb, 512 / (int)kTrsmTmemCols);
  return std::max(nb, 1);
}

}  // namespace feti
