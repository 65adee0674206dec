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

#include "common.cuh"
#include "kernels.h"

namespace feti {
namespace {

__device__ __forceinline__ int pop_item(int* queue) {
  __shared__ int item;
  __syncthreads();
  if (threadIdx.x == 0) item = atomicAdd(queue, 1);
  __syncthreads();
  return item;
}

// acc[a][b] += sum_k A[k][ty + 16a] * B[k][tx + 16b]
__device__ __forceinline__ void tile_mma(const double (*A)[kT], const double (*B)[kT], int kc,
                                         double acc[4][4], int tx, int ty) {
  for (int k = 0; k < kc; ++k) {
    double a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = A[k][ty + 16 * u];
      b[u] = B[k][tx + 16 * u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
  }
}

struct Smem {
  double D[kNB][kNB + 1];
  double A[kNB][kT];
  double B[kNB][kT];
  double red[kThreads / 32];
};

// Unblocked Cholesky of the nbk x nbk block in sm.D (lower).  Sets *bad on a
// non-positive pivot (the pivot is then replaced by 1 so the sweep finishes).
__device__ void chol_diag(Smem& sm, int nbk, int* bad) {
  const int tid = threadIdx.x;
  for (int k = 0; k < nbk; ++k) {
    if (tid == 0) {
      double d = sm.D[k][k];
      if (!(d > 0.0)) {
        *bad = 1;
        d = 1.0;
      }
      sm.D[k][k] = sqrt(d);
    }
    __syncthreads();
    if (tid > k && tid < nbk) sm.D[tid][k] = sm.D[tid][k] / sm.D[k][k];
    __syncthreads();
    int rem = nbk - k - 1;
    for (int idx = tid; idx < rem * rem; idx += kThreads) {
      int i = k + 1 + idx % rem, j = k + 1 + idx / rem;
      if (i >= j) sm.D[i][j] -= sm.D[i][k] * sm.D[j][k];
    }
    __syncthreads();
  }
}

// Partial dense factorisation of one front: eliminate the first w columns of
// the (w+r) x (w+r) symmetric front held as Ls (column-major f x w) and W
// (column-major r x r, lower part used).
__device__ void factor_front(Smem& sm, double* Ls, int f, int w, double* W, int r, int* bad) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  for (int kb = 0; kb < w; kb += kNB) {
    const int nbk = min(kNB, w - kb);
    for (int idx = tid; idx < kNB * kNB; idx += kThreads) {
      int i = idx % kNB, j = idx / kNB;
      sm.D[i][j] = (i < nbk && j <= i) ? Ls[(int64_t)(kb + j) * f + kb + i] : 0.0;
    }
    __syncthreads();
    chol_diag(sm, nbk, bad);
    for (int idx = tid; idx < nbk * nbk; idx += kThreads) {
      int i = idx % nbk, j = idx / nbk;
      if (i >= j) Ls[(int64_t)(kb + j) * f + kb + i] = sm.D[i][j];
    }
    // panel: rows below the block, L_ib = A_ib L_bb^{-T}
    const int i0 = kb + nbk;
    for (int i = i0 + tid; i < f; i += kThreads) {
      double x[kNB];
#pragma unroll
      for (int k = 0; k < kNB; ++k) x[k] = (k < nbk) ? Ls[(int64_t)(kb + k) * f + i] : 0.0;
#pragma unroll
      for (int k = 0; k < kNB; ++k) {
        if (k < nbk) {
          double s = x[k];
#pragma unroll
          for (int l = 0; l < k; ++l) s = fma(-sm.D[k][l], x[l], s);
          x[k] = s / sm.D[k][k];
        }
      }
#pragma unroll
      for (int k = 0; k < kNB; ++k)
        if (k < nbk) Ls[(int64_t)(kb + k) * f + i] = x[k];
    }
    __syncthreads();
    // trailing update C -= L_ib L_jb^T on the lower triangle of rows/cols [i0, f)
    const int nr = f - i0;
    const int T = (nr + kT - 1) / kT;
    for (int ti = 0; ti < T; ++ti) {
      for (int tj = 0; tj <= ti; ++tj) {
        const int ri = i0 + ti * kT, cj = i0 + tj * kT;
        for (int idx = tid; idx < nbk * kT; idx += kThreads) {
          int x = idx % kT, k = idx / kT;
          const double* col = Ls + (int64_t)(kb + k) * f;
          sm.A[k][x] = (ri + x < f) ? col[ri + x] : 0.0;
          sm.B[k][x] = (cj + x < f) ? col[cj + x] : 0.0;
        }
        __syncthreads();
        double acc[4][4] = {};
        tile_mma(sm.A, sm.B, nbk, acc, tx, ty);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          int i = ri + ty + 16 * u;
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            int j = cj + tx + 16 * v;
            if (i < f && j <= i) {
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

__global__ void __launch_bounds__(kThreads) chol_kernel(DevPlan P, const int* order, int nsub, int* queue,
                                                         double* ws, int64_t ws_stride, int64_t front_sz,
                                                         int* status) {
  __shared__ Smem sm;
  __shared__ int bad;
  const int tid = threadIdx.x;
  double* W = ws + (int64_t)blockIdx.x * ws_stride;
  double* stack = W + front_sz;
  for (;;) {
    int it = pop_item(queue);
    if (it >= nsub) return;
    const int si = order[it];
    const SubInfo S = P.sub[si];
    const double* K = P.Kval + S.Kval;
    double* L = P.L + S.L;
    if (tid == 0) bad = 0;
    // rho = max diag K_i (fixing-node penalty)
    double mx = 0.0;
    for (int i = tid; i < S.n; i += kThreads) mx = fmax(mx, K[P.diag_src[S.diag0 + i]]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) sm.red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
      double m2 = sm.red[0];
      for (int k = 1; k < kThreads / 32; ++k) m2 = fmax(m2, sm.red[k]);
      sm.red[0] = m2;
      P.rho[si] = m2;
    }
    __syncthreads();
    const double rho = sm.red[0];
    for (int s = 0; s < S.nsn; ++s) {
      const int gs = S.sn0 + s;
      const int w = P.sn_w[gs], r = P.sn_r[gs], f = w + r;
      double* Ls = L + P.Lofs[gs];
      for (int64_t idx = tid; idx < (int64_t)f * w; idx += kThreads) Ls[idx] = 0.0;
      for (int64_t idx = tid; idx < (int64_t)r * r; idx += kThreads) W[idx] = 0.0;
      __syncthreads();
      for (int64_t k = P.kmap_off[gs] + tid; k < P.kmap_off[gs + 1]; k += kThreads)
        L[P.kmap_dst[k]] = K[P.kmap_src[k]];
      __syncthreads();
      if (tid < S.nfix && P.fix_sn[S.fix0 + tid] == s) L[P.fix_pos[S.fix0 + tid]] += rho;
      for (int c = P.ch_off[gs]; c < P.ch_off[gs + 1]; ++c) {
        const int gc = S.sn0 + P.ch_list[c];
        const int rc = P.sn_r[gc];
        const double* U = stack + P.upd_ofs[gc];
        const int* rl = P.rel + P.rel_off[gc];
        __syncthreads();
        for (int64_t idx = tid; idx < (int64_t)rc * rc; idx += kThreads) {
          int a = (int)(idx % rc), b = (int)(idx / rc);
          if (a < b) continue;
          int ra = rl[a], rb = rl[b];
          double v = U[idx];
          if (rb < w) Ls[(int64_t)rb * f + ra] += v;
          else W[(int64_t)(rb - w) * r + (ra - w)] += v;
        }
      }
      __syncthreads();
      factor_front(sm, Ls, f, w, W, r, &bad);
      __syncthreads();
      if (P.sn_parent[gs] >= 0) {
        double* dst = stack + P.upd_ofs[gs];
        for (int64_t idx = tid; idx < (int64_t)r * r; idx += kThreads) dst[idx] = W[idx];
      }
      __syncthreads();
    }
    if (tid == 0 && bad) atomicOr(status, kStatNotSPD);
  }
}

// Smem of the solve (element type T of X).
template <typename T>
struct SolveSmem {
  T D[kNB][kNB + 1];
  T A[kNB][kT];
  T B[kNB][kT];
};

// Forward solve of one RHS front: X_s = L_ss^{-1} X_s, then C -= L_rs X_s
// (C = the r bottom rows).  Column-major fronts: column j of X_s is
// Xs[j * wp + 0 .. w), column j of the bottom block is W2[j * r + 0 .. r).
template <typename T>
__device__ void solve_front(SolveSmem<T>& sm, const double* Ls, int f, int w, T* Xs, int wp, T* W2, int J) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int r = f - w;
  for (int kb = 0; kb < w; kb += kNB) {
    const int nbk = min(kNB, w - kb);
    for (int idx = tid; idx < kNB * kNB; idx += kThreads) {
      int i = idx % kNB, j = idx / kNB;
      sm.D[i][j] = (i < nbk && j <= i) ? (T)Ls[(int64_t)(kb + j) * f + kb + i] : (T)0;
    }
    __syncthreads();
    for (int col = tid; col < J; col += kThreads) {
      T* xc = Xs + (int64_t)col * wp + kb;
      T x[kNB];
#pragma unroll
      for (int k = 0; k < kNB; ++k) x[k] = (k < nbk) ? xc[k] : (T)0;
#pragma unroll
      for (int k = 0; k < kNB; ++k) {
        if (k < nbk) {
          T s = x[k];
#pragma unroll
          for (int l = 0; l < k; ++l) s = fma(-sm.D[k][l], x[l], s);
          x[k] = s / sm.D[k][k];
        }
      }
#pragma unroll
      for (int k = 0; k < kNB; ++k)
        if (k < nbk) xc[k] = x[k];
    }
    __syncthreads();
    const int i0 = kb + nbk;
    const int TR = (f - i0 + kT - 1) / kT, TC = (J + kT - 1) / kT;
    for (int ti = 0; ti < TR; ++ti) {
      for (int tc = 0; tc < TC; ++tc) {
        const int ri = i0 + ti * kT, cj = tc * kT;
        for (int idx = tid; idx < nbk * kT; idx += kThreads) {
          int x = idx % kT, k = idx / kT;
          sm.A[k][x] = (ri + x < f) ? (T)Ls[(int64_t)(kb + k) * f + ri + x] : (T)0;
        }
        for (int idx = tid; idx < kNB * kT; idx += kThreads) {
          int k = idx % kNB, y = idx / kNB;
          sm.B[k][y] = (k < nbk && cj + y < J) ? Xs[(int64_t)(cj + y) * wp + kb + k] : (T)0;
        }
        __syncthreads();
        T acc[4][4] = {};
        for (int k = 0; k < nbk; ++k) {
          T a[4], b[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            a[u] = sm.A[k][tx + 16 * u];
            b[u] = sm.B[k][ty + 16 * u];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          int col = cj + ty + 16 * v;
          if (col >= J) continue;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            int i = ri + tx + 16 * u;
            if (i >= f) continue;
            if (i < w) Xs[(int64_t)col * wp + i] -= acc[u][v];
            else W2[(int64_t)col * r + (i - w)] -= acc[u][v];
          }
        }
        __syncthreads();
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) trsm_kernel(DevPlan P, const int* order, int nsub, int* queue,
                                                         T* X, T* ws, int64_t ws_stride, int64_t front_sz) {
  __shared__ SolveSmem<T> sm;
  const int tid = threadIdx.x;
  T* W2 = ws + (int64_t)blockIdx.x * ws_stride;
  T* stack = W2 + front_sz;
  for (;;) {
    int it = pop_item(queue);
    if (it >= nsub) return;
    const int si = order[it];
    const SubInfo S = P.sub[si];
    const double* L = P.L + S.L;
    T* Xsub = X + S.X;
    for (int a = 0; a < S.nact; ++a) {
      const int s = P.act[S.act0 + a];
      const int gs = S.sn0 + s, bs = S.bsn0 + s;
      const int c0 = P.sn_c0[gs], w = P.sn_w[gs], r = P.sn_r[gs], f = w + r;
      const int wp = (w + 3) & ~3;
      const int jb = P.jb[bs], je = P.je[bs], jo = P.jo[bs];
      const int J = je - jb;
      T* Xs = Xsub + P.Xofs[bs];
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
        const int Jc = P.je[bc] - P.jb[bc];
        if (Jc <= 0) continue;
        const int rc = P.sn_r[gc], coff = P.jb[bc] - jb;
        const T* U = stack + P.rhs_ofs[bc];
        const int* rl = P.rel + P.rel_off[gc];
        // children own disjoint column ranges: no conflicts between them
        for (int64_t idx = tid; idx < (int64_t)rc * Jc; idx += kThreads) {
          int col = (int)(idx / rc), a2 = (int)(idx % rc);
          int ra = rl[a2];
          T v = U[idx];
          if (ra < w) Xs[(int64_t)(coff + col) * wp + ra] += v;
          else W2[(int64_t)(coff + col) * r + (ra - w)] += v;
        }
      }
      __syncthreads();
      solve_front<T>(sm, L + P.Lofs[gs], f, w, Xs, wp, W2, J);
      __syncthreads();
      if (P.sn_parent[gs] >= 0) {
        T* dst = stack + P.rhs_ofs[bs];
        for (int64_t idx = tid; idx < (int64_t)r * J; idx += kThreads) dst[idx] = W2[idx];
      }
      __syncthreads();
    }
  }
}

}  // namespace

void launch_chol(const DevPlan& P, const int* order, int nsub, int* queue, double* ws, int64_t ws_stride,
                 int64_t front_sz, int grid, int* status, cudaStream_t st) {
  chol_kernel<<<grid, kThreads, 0, st>>>(P, order, nsub, queue, ws, ws_stride, front_sz, status);
}

void launch_trsm(const DevPlan& P, const int* order, int nsub, int* queue, void* X, bool fp32, double* ws,
                 int64_t ws_stride, int64_t front_sz, int grid, cudaStream_t st) {
  if (fp32)
    trsm_kernel<float><<<grid, kThreads, 0, st>>>(P, order, nsub, queue, (float*)X, (float*)ws, 2 * ws_stride,
                                                  front_sz);
  else
    trsm_kernel<double><<<grid, kThreads, 0, st>>>(P, order, nsub, queue, (double*)X, ws, ws_stride, front_sz);
}

}  // namespace feti
