// FP64 SIMT SYRK F_i = X_i^T X_i into lower F tiles (paper Sec. IV, SYRK
// path; the mixed-precision path uses the tensor-core kernel instead).
//
// F_i layout (common.cuh): the m_pad x m_pad matrix (columns in sorted
// order) is cut into kT x kT tiles; only tiles (bi, bj) with bj <= bi are
// stored, tile index bi (bi + 1) / 2 + bj.  Off-diagonal tiles are row-major;
// diagonal tiles keep only the 16-byte chunks of each row up to the diagonal.
#include "common.cuh"
#include "kernels.h"

namespace feti {
namespace {

__device__ __forceinline__ void tile_of(int t, int& bi, int& bj) {
  int b = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((b + 1) * (b + 2) / 2 <= t) ++b;
  while (b * (b + 1) / 2 > t) --b;
  bi = b;
  bj = t - b * (b + 1) / 2;
}

// ---------------------------------------------------------------- FP64 SYRK

__global__ void __launch_bounds__(kThreads) syrk_f64_kernel(DevPlan P, const int2* items, int nitems,
                                                            const double* X, double* F) {
  __shared__ double A[32][kT];
  __shared__ double B[32][kT];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int si = items[it].x, t = items[it].y;
    const SubInfo S = P.sub[si];
    int bi, bj;
    tile_of(t, bi, bj);
    double acc[4][4] = {};
    const int* tl = P.tile_off + S.tile0;
    for (int c = tl[t]; c < tl[t + 1]; ++c) {
      const int s = P.tile_sn[c];
      const int gs = S.sn0 + s, bs = S.bsn0 + s;
      const int w = P.sn_w[gs], wp = (w + 7) & ~7, jb = P.jb[bs], J = P.je[bs] - jb;
      const double* Xs = X + S.X + P.Xofs[bs];
      const int ca = bi * kT - jb, cb = bj * kT - jb;
      for (int k0 = 0; k0 < w; k0 += 32) {
        const int kc = min(32, w - k0);
        for (int idx = tid; idx < 32 * kT; idx += kThreads) {
          int k = idx % 32, x = idx / 32;
          bool kin = k < kc;
          int xa = ca + x, xb = cb + x;
          A[k][x] = (kin && xa >= 0 && xa < J) ? Xs[(int64_t)xa * wp + k0 + k] : 0.0;
          B[k][x] = (kin && xb >= 0 && xb < J) ? Xs[(int64_t)xb * wp + k0 + k] : 0.0;
        }
        __syncthreads();
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
        __syncthreads();
      }
    }
    double* Ft = F + S.F + tile_offset<8>(S.nb, S.vr, bi, bj);
    const int nrow = tile_rows(S.nb, S.vr, bi);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int r = ty + 16 * u, c = tx + 16 * v;
        if (r >= nrow) continue;
        if (bj < bi) Ft[tile_pos(r, c)] = acc[u][v];
        else if (c / 2 <= r / 2) Ft[diag_pos<8>(r, c)] = c <= r ? acc[u][v] : 0.0;  // diagonal tile
      }
  }
}

// unpack F_i (sorted order) to a dense m x m in B-row order (test helper)
template <typename TF>
__global__ void unpack_F_kernel(const TF* Fsub, int m, int nb, int vr, const int* colperm, double* out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < (int64_t)m * m; g += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(g / m), j = (int)(g % m);
    if (j / kT > i / kT || (j / kT == i / kT && j % kT > i % kT)) {  // F is symmetric: read the lower copy
      int t = i;
      i = j;
      j = t;
    }
    constexpr int E = (int)sizeof(TF);
    const int64_t o = tile_offset<E>(nb, vr, i / kT, j / kT);
    const double v = (double)Fsub[o + (i / kT == j / kT ? diag_pos<E>(i % kT, j % kT) : tile_pos(i % kT, j % kT))];
    out[(int64_t)colperm[(int)(g / m)] * m + colperm[(int)(g % m)]] = v;
  }
}

// M_i tiles in the layout and sorted column order of F_i from the Schur complement S_i that an unfactored
// root front holds (the DOFs B touches ordered last): M[a][b] = s_a s_b S[t_a][t_b], with t the position of
// column a's DOF in the root block and s_a the sign of B in that column.  M_i = B_i S_i B_i^T restricted to
// the subdomain's multipliers, the local block of the Dirichlet preconditioner.
template <typename TF>
__global__ void schur_tiles_kernel(DevPlan P, const TileDesc* desc, int ntiles, TF* M) {
  constexpr int E = (int)sizeof(TF), V = 16 / E;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const TileDesc d = desc[t];
    const bool diag = (d.flags & kTileDiag) != 0;
    const SubInfo& S = P.sub[P.colsub[d.prow]];
    const int gr = S.sn0 + S.nsn - 1;
    const int c0 = P.sn_c0[gr], f = P.sn_w[gr] + P.sn_r[gr];
    const double* Ls = P.L + S.L + P.Lofs[gr];
    const int* iperm = P.iperm + S.diag0;
    TF* Mt = M + d.f_ofs;
    for (int idx = threadIdx.x; idx < d.rows * kT; idx += blockDim.x) {
      const int r = idx / kT, cc = idx % kT;
      if (diag && cc >= V * ((r + V) / V)) continue;  // not stored
      const int a = d.prow + r, b = d.pcol + cc;
      double v = 0.0;
      if (!(diag && cc > r) && P.qmap[a] >= 0 && P.qmap[b] >= 0) {
        const int ia = iperm[P.qdof[a]] - c0, ib = iperm[P.qdof[b]] - c0;
        const int hi = max(ia, ib), lo = min(ia, ib);
        v = P.qsign[a] * P.qsign[b] * Ls[(int64_t)lo * f + hi];
      }
      Mt[diag ? diag_pos<E>(r, cc) : tile_pos(r, cc)] = (TF)v;
    }
  }
}

}  // namespace

void launch_schur_tiles(const DevPlan& P, const TileDesc* desc, int ntiles, bool fp32, void* M, int grid,
                        cudaStream_t st) {
  if (ntiles <= 0) return;
  if (fp32) schur_tiles_kernel<float><<<grid, 256, 0, st>>>(P, desc, ntiles, (float*)M);
  else schur_tiles_kernel<double><<<grid, 256, 0, st>>>(P, desc, ntiles, (double*)M);
}

void launch_syrk_f64(const DevPlan& P, const int2* items, int nitems, const double* X, double* F, int grid,
                     cudaStream_t st) {
  syrk_f64_kernel<<<grid, kThreads, 0, st>>>(P, items, nitems, X, F);
}

void launch_unpack_F(const void* Fsub, bool fp32, int m, int nb, int vr, const int* colperm, double* out,
                     cudaStream_t st) {
  int64_t tot = (int64_t)m * m;
  int grid = (int)std::min<int64_t>((tot + 255) / 256, 4096);
  if (grid < 1) grid = 1;
  if (fp32) unpack_F_kernel<float><<<grid, 256, 0, st>>>((const float*)Fsub, m, nb, vr, colperm, out);
  else unpack_F_kernel<double><<<grid, 256, 0, st>>>((const double*)Fsub, m, nb, vr, colperm, out);
}

}  // namespace feti
