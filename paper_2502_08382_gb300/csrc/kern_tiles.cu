// SYRK F_i = X_i^T X_i into lower F tiles, and the explicit application
// q = sum_i B~_i^T F_i B~_i p (paper eq. 12 and Algorithm 2's
// scatter / apply / gather) as a packed-tile SYMV.
//
// F_i layout: the m_pad x m_pad matrix (columns in sorted order) is cut into
// kT x kT tiles; only tiles (bi, bj) with bj <= bi are stored, tile index
// bi (bi + 1) / 2 + bj, each tile row-major.  Diagonal tiles are stored in
// full (both triangles), so one tile is one contiguous 16/32 KB block.
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
      const int w = P.sn_w[gs], wp = (w + 3) & ~3, jb = P.jb[bs], J = P.je[bs] - jb;
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
    double* Ft = F + S.F + (int64_t)t * kT * kT;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) Ft[(ty + 16 * u) * kT + tx + 16 * v] = acc[u][v];
  }
}

// ---------------------------------------------------------------- apply, phase 1
// One CTA per (subdomain, tile row b): row partial of block b over the tiles
// (b, 0..b), and the transposed partial of each off-diagonal tile (b, bj)
// which belongs to block bj (written to tpart, summed in phase 2).

template <typename TF>
__global__ void __launch_bounds__(kThreads) apply_rows_kernel(DevPlan P, const int2* items, int nitems,
                                                              const TF* F, const double* p, double* trow,
                                                              double* tpart) {
  __shared__ TF Fs[kT][kT + 1];
  __shared__ double pb[kT], pj[kT];
  __shared__ double racc[4][kT];
  const int tid = threadIdx.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int si = items[it].x, b = items[it].y;
    const SubInfo S = P.sub[si];
    if (tid < kT) {
      int lam = P.qmap[S.qcol + b * kT + tid];
      pb[tid] = lam >= 0 ? p[lam] : 0.0;
    }
    double rsum = 0.0;
    const int rr = tid % kT, part = tid / kT;  // 4 threads share a row
    for (int bj = 0; bj <= b; ++bj) {
      const int t = b * (b + 1) / 2 + bj;
      const TF* Ft = F + S.F + (int64_t)t * kT * kT;
      __syncthreads();
      if (tid < kT) {
        int lam = P.qmap[S.qcol + bj * kT + tid];
        pj[tid] = lam >= 0 ? p[lam] : 0.0;
      }
      for (int idx = tid; idx < kT * kT; idx += kThreads) Fs[idx / kT][idx % kT] = Ft[idx];
      __syncthreads();
      // row partial: 4 threads per row, 16 columns each
      double s = 0.0;
#pragma unroll 4
      for (int c = part * 16; c < part * 16 + 16; ++c) s += (double)Fs[rr][c] * pj[c];
      rsum += s;
      if (bj < b) {
        // column partial: F_t^T p_b, 4 threads per column, 16 rows each
        double cs = 0.0;
#pragma unroll 4
        for (int r2 = part * 16; r2 < part * 16 + 16; ++r2) cs += (double)Fs[r2][rr] * pb[r2];
        racc[part][rr] = cs;
        __syncthreads();
        if (tid < kT)
          tpart[S.tpart + (int64_t)t * kT + tid] = racc[0][tid] + racc[1][tid] + racc[2][tid] + racc[3][tid];
      }
    }
    __syncthreads();
    racc[part][rr] = rsum;
    __syncthreads();
    if (tid < kT) trow[S.trow + b * kT + tid] = racc[0][tid] + racc[1][tid] + racc[2][tid] + racc[3][tid];
    __syncthreads();
  }
}

// phase 2: q_i[j] = trow[j] + sum_{bi > b(j)} tpart[(bi, b(j))][j mod kT]
__global__ void apply_cols_kernel(DevPlan P, const int* colsub, int64_t ncols, const double* trow,
                                  const double* tpart, double* qi) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ncols; g += (int64_t)gridDim.x * blockDim.x) {
    const int si = colsub[g];
    const SubInfo S = P.sub[si];
    const int j = (int)(g - S.qcol);
    const int b = j / kT, l = j % kT;
    double s = trow[g];
    for (int bi = b + 1; bi < S.nb; ++bi) s += tpart[S.tpart + (int64_t)(bi * (bi + 1) / 2 + b) * kT + l];
    qi[g] = s;
  }
}

// phase 3: q[lambda] = sum of its (at most two) subdomain contributions, fixed order
__global__ void gather_lambda_kernel(const int* c0, const int* c1, int nlam, const double* qi, double* q) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlam; l += gridDim.x * blockDim.x) {
    int a = c0[l], b = c1[l];
    double s = a >= 0 ? qi[a] : 0.0;
    if (b >= 0) s += qi[b];
    q[l] = s;
  }
}

// unpack F_i (sorted order) to a dense m x m in B-row order (test helper)
template <typename TF>
__global__ void unpack_F_kernel(const TF* Fsub, int m, int nb, const int* colperm, double* out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < (int64_t)m * m; g += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(g / m), j = (int)(g % m);
    int bi = i / kT, bj = j / kT;
    double v;
    if (bj <= bi) v = (double)Fsub[(int64_t)(bi * (bi + 1) / 2 + bj) * kT * kT + (i % kT) * kT + (j % kT)];
    else v = (double)Fsub[(int64_t)(bj * (bj + 1) / 2 + bi) * kT * kT + (j % kT) * kT + (i % kT)];
    out[(int64_t)colperm[i] * m + colperm[j]] = v;
  }
}

}  // namespace

void launch_syrk_f64(const DevPlan& P, const int2* items, int nitems, const double* X, double* F, int grid,
                     cudaStream_t st) {
  syrk_f64_kernel<<<grid, kThreads, 0, st>>>(P, items, nitems, X, F);
}

void launch_apply_rows_f64(const DevPlan& P, const int2* items, int nitems, const double* F, const double* p,
                           double* trow, double* tpart, int grid, cudaStream_t st) {
  apply_rows_kernel<double><<<grid, kThreads, 0, st>>>(P, items, nitems, F, p, trow, tpart);
}

void launch_apply_rows_f32(const DevPlan& P, const int2* items, int nitems, const float* F, const double* p,
                           double* trow, double* tpart, int grid, cudaStream_t st) {
  apply_rows_kernel<float><<<grid, kThreads, 0, st>>>(P, items, nitems, F, p, trow, tpart);
}

void launch_apply_cols(const DevPlan& P, const int* colsub, int64_t ncols, const double* trow,
                       const double* tpart, double* qi, cudaStream_t st) {
  int grid = (int)std::min<int64_t>((ncols + 255) / 256, 152 * 16);
  apply_cols_kernel<<<grid, 256, 0, st>>>(P, colsub, ncols, trow, tpart, qi);
}

void launch_gather_lambda(const int* c0, const int* c1, int nlam, const double* qi, double* q, cudaStream_t st) {
  int grid = std::min((nlam + 255) / 256, 152 * 16);
  gather_lambda_kernel<<<grid, 256, 0, st>>>(c0, c1, nlam, qi, q);
}

void launch_unpack_F(const void* Fsub, bool fp32, int m, int nb, const int* colperm, double* out, cudaStream_t st) {
  int64_t tot = (int64_t)m * m;
  int grid = (int)std::min<int64_t>((tot + 255) / 256, 4096);
  if (grid < 1) grid = 1;
  if (fp32) unpack_F_kernel<float><<<grid, 256, 0, st>>>((const float*)Fsub, m, nb, colperm, out);
  else unpack_F_kernel<double><<<grid, 256, 0, st>>>((const double*)Fsub, m, nb, colperm, out);
}

}  // namespace feti
