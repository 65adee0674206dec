// FP64 adjoint of the weighted trace L = sum_i <W_i, F_i> and the trace itself.
//
// dL/dtheta_e = -<Z^T dK_e Z, W> for Z = K_reg^{-1} B^T (derivative of the
// inverse, rho held fixed).  After the assembly L is kept in unit-lower form,
// L = L_u D, so K_reg^{-1} = P^T L_u^{-T} D^{-2} L_u^{-1} P and, with the pruned
// forward solve X_u = L_u^{-1} P B^T (staircase blocks X_s, w_s x J_s):
//   Z = P^T L_u^{-T} D^{-2} X_u,   Y = Z W = P^T L_u^{-T} D^{-2} (X_u W),
//   dL/dtheta_e = -sum_{a,b in e} (dK_e)_ab Y[b,:] . Z[a,:].
// Forming Y from X_u W (2 nnz(X_u) m flops) and one backward solve is several
// times cheaper than the dense product Z W (2 n m^2 flops).  The kernels work
// on a batch of subdomains whose dense arrays V = [D^{-2} X_u | D^{-2} X_u W]
// (n x 2 m_pad, row-major, rows in the factor's numbering) fit the buffer:
//   adj_build_kernel   V_Z rows from X_u, V_Y = X_u W per active supernode
//   adj_bsolve_kernel  V <- L_u^{-T} V, one CTA per 64 columns of a subdomain,
//                      supernodes from the root down
//   adj_contract_kernel per element, the 24 x 24 (or smaller) contraction.
// Everything is FP64 (the adjoint is an FP64 kernel by design).
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace feti {
namespace {

constexpr int kAT = 256;   // threads per CTA
constexpr int kCB = 64;    // columns per bsolve item

__device__ __forceinline__ int pop(int* queue) {
  __shared__ int item;
  __syncthreads();
  if (threadIdx.x == 0) item = atomicAdd(queue, 1);
  __syncthreads();
  return item;
}

// Ws[a][b] = W[cp[a]][cp[b]] in sorted column order, zero beyond m (m_pad x m_pad)
__global__ void wsort_kernel(const AdjBatch* B, int nb, const double* W, const int* colperm, double* work) {
  const AdjBatch& E = B[blockIdx.y];
  const int m = E.m, mp = E.m_pad;
  const int* cp = colperm + E.qcol;
  const double* Wi = W + E.w_src;
  double* Ws = work + E.ws_ofs;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < (int64_t)mp * mp;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(g / mp), b = (int)(g % mp);
    Ws[g] = (a < m && b < m) ? Wi[(int64_t)cp[a] * m + cp[b]] : 0.0;
  }
}

// One item = (batch entry, active supernode s, 64-row block k0 of its own rows,
// column group cg of kBuildCols columns):
//   V_Z[c0 + k][jb + j] = d2[c0 + k] X_s[j][k]            (j < J_s; written by column group 0)
//   V_Y[c0 + k][c]      = d2[c0 + k] sum_j X_s[j][k] Ws[jb + j][c]
// computed in 64 x 64 output tiles (4 x 4 per thread) over 32-deep chunks of j.
__global__ void __launch_bounds__(kAT) adj_build_kernel(DevPlan P, const AdjBatch* B, const int4* items, int nitems,
                                                       int* queue, const double* Xu, double* work) {
  __shared__ double As[32][kT + 1];  // X chunk: [j][k]
  __shared__ double Bs[32][kT];      // Ws chunk: [j][c]
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  for (;;) {
    const int it = pop(queue);
    if (it >= nitems) return;
    const int4 item = items[it];
    const AdjBatch& E = B[item.x];
    const SubInfo& S = P.sub[E.sub];
    const int s = P.act[S.act0 + item.y];
    const int gs = S.sn0 + s, bs = S.bsn0 + s;
    const int c0 = P.sn_c0[gs], w = P.sn_w[gs], wp = (w + 7) & ~7;
    const int jb = P.jb[bs], J = P.je[bs] - jb;
    const double* Xs = Xu + S.X + P.Xofs[bs];
    const double* d2 = P.dinv + S.dof;
    const int mp = E.m_pad;
    const int64_t ld = (E.zonly ? 1 : 2) * (int64_t)mp;
    double* V = work + E.v_ofs;
    const double* Ws = work + E.ws_ofs;
    const int k0 = item.z, nk = min(kT, w - k0);
    if (item.w == 0)
      for (int64_t idx = tid; idx < (int64_t)nk * J; idx += kAT) {
        const int k = (int)(idx % nk), j = (int)(idx / nk);
        V[(int64_t)(c0 + k0 + k) * ld + jb + j] = d2[c0 + k0 + k] * Xs[(int64_t)j * wp + k0 + k];
      }
    const int cend = E.zonly ? 0 : min(mp, item.w + kBuildCols);
    for (int cb = item.w; cb < cend; cb += kT) {
      double acc[4][4] = {};
      for (int j0 = 0; j0 < J; j0 += 32) {
        __syncthreads();
        for (int idx = tid; idx < 32 * kT; idx += kAT) {
          const int j = idx / kT, k = idx % kT;
          As[j][k] = (j0 + j < J && k < nk) ? Xs[(int64_t)(j0 + j) * wp + k0 + k] : 0.0;
          Bs[j][k] = (j0 + j < J) ? Ws[(int64_t)(jb + j0 + j) * mp + cb + k] : 0.0;
        }
        __syncthreads();
        const int jn = min(32, J - j0);
        for (int j = 0; j < jn; ++j) {
          double a[4], b[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) a[u] = As[j][ty + 16 * u];
#pragma unroll
          for (int v = 0; v < 4; ++v) b[v] = Bs[j][tx + 16 * v];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = ty + 16 * u;
        if (k >= nk) continue;
        const double sc = d2[c0 + k0 + k];
        double* row = V + (int64_t)(c0 + k0 + k) * ld + mp + cb;
#pragma unroll
        for (int v = 0; v < 4; ++v) row[tx + 16 * v] = sc * acc[u][v];
      }
    }
  }
}

// V <- L_u^{-T} V for the 64 columns [cb, cb + 64) of one batch entry's V.
// Supernodes from the root down (reverse postorder); within a supernode the
// own columns in 32-wide blocks from the last one: the block's rows take
//   V_b -= L[below, b]^T V[below]   (below = later own rows, then struct rows)
// as a GEMM over 32-row chunks, then the unit upper-triangular solve with the
// block's own 32 x 32 triangle (four threads per column, warp reductions).
__global__ void __launch_bounds__(kAT) adj_bsolve_kernel(DevPlan P, const AdjBatch* B, const int2* items, int nitems,
                                                        int* queue, double* work) {
  __shared__ double Lc[32][33];      // L chunk: [k][i]
  __shared__ double Vc[32][kCB];     // V chunk: [i][c]
  __shared__ double Xb[32][kCB];     // the block's rows being solved
  __shared__ int rowid[32];
  const int tid = threadIdx.x;
  const int c = tid % kCB, kg = tid / kCB;  // GEMM: column c, rows kg * 8 .. + 7
  for (;;) {
    const int it = pop(queue);
    if (it >= nitems) return;
    const AdjBatch& E = B[items[it].x];
    const SubInfo& S = P.sub[E.sub];
    const int cb = items[it].y * kCB;
    const int64_t ld = (E.zonly ? 1 : 2) * (int64_t)E.m_pad;
    double* V = work + E.v_ofs + cb;
    const double* Lsub = P.L + S.L;
    for (int s = S.nsn - 1; s >= 0; --s) {
      const int gs = S.sn0 + s;
      const int c0 = P.sn_c0[gs], w = P.sn_w[gs], r = P.sn_r[gs], f = w + r;
      const double* Ls = Lsub + P.Lofs[gs];
      const int* srow = P.rows + P.sn_rows[gs];
      for (int kb = ((w - 1) / 32) * 32; kb >= 0; kb -= 32) {
        const int nbk = min(32, w - kb);
        double acc[8] = {};
        for (int i0 = kb + nbk; i0 < f; i0 += 32) {
          const int ni = min(32, f - i0);
          __syncthreads();
          if (tid < 32) rowid[tid] = tid < ni ? (i0 + tid < w ? c0 + i0 + tid : srow[i0 + tid - w]) : -1;
          for (int idx = tid; idx < 32 * 32; idx += kAT) {
            const int k = idx / 32, i = idx % 32;
            Lc[k][i] = (k < nbk && i < ni) ? Ls[(int64_t)(kb + k) * f + i0 + i] : 0.0;
          }
          __syncthreads();
          for (int idx = tid; idx < 32 * kCB; idx += kAT) {
            const int i = idx / kCB, cc = idx % kCB;
            Vc[i][cc] = i < ni ? V[(int64_t)rowid[i] * ld + cc] : 0.0;
          }
          __syncthreads();
          for (int i = 0; i < ni; ++i) {
            const double v = Vc[i][c];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = fma(Lc[kg * 8 + u][i], v, acc[u]);
          }
        }
        __syncthreads();
        // the block's rows minus the update; the block's own triangle into Lc
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k = kg * 8 + u;
          Xb[k][c] = k < nbk ? V[(int64_t)(c0 + kb + k) * ld + c] - acc[u] : 0.0;
        }
        for (int idx = tid; idx < 32 * 32; idx += kAT) {
          const int k = idx / 32, i = idx % 32;
          Lc[k][i] = (k < nbk && i < nbk && i > k) ? Ls[(int64_t)(kb + k) * f + kb + i] : 0.0;
        }
        __syncthreads();
        {
          // unit upper solve L_bb^T x = Xb: column cc by the four lanes 4 cc' .. 4 cc' + 3 of one warp
          const int col = tid / 4, part = tid % 4;
          for (int k = nbk - 1; k >= 0; --k) {
            double sum = 0.0;
            for (int i = k + 1 + part; i < nbk; i += 4) sum = fma(Lc[k][i], Xb[i][col], sum);
            sum += __shfl_xor_sync(0xffffffffu, sum, 1);
            sum += __shfl_xor_sync(0xffffffffu, sum, 2);
            if (part == 0) Xb[k][col] -= sum;
            __syncwarp();
          }
        }
        __syncthreads();
        for (int idx = tid; idx < nbk * kCB; idx += kAT) {
          const int k = idx / kCB, cc = idx % kCB;
          V[(int64_t)(c0 + kb + k) * ld + cc] = Xb[k][cc];
        }
      }
    }
  }
}

// g[e] = -scale_e sum_{a,b} dK_e[a][b] (Y[b,:] . Z[a,:]) with Z row a = V_Z[iperm[dof_a]],
// Y row b = V_Y[iperm[dof_b]]; one CTA per element at a time, 32-wide chunks of the columns.
constexpr int kKW = 32;
__global__ void __launch_bounds__(kAT) adj_contract_kernel(DevPlan P, const AdjBatch* B, int nb, const int* eldofs,
                                                          const double* eldk, const double* elsc, const double* work,
                                                          double* g) {
  __shared__ double Zs[32][kKW + 1];
  __shared__ double Ys[32][kKW + 1];
  __shared__ int ridx[32];
  __shared__ double red[kAT / 32];
  const int tid = threadIdx.x;
  const AdjBatch& E = B[blockIdx.y];
  const SubInfo& S = P.sub[E.sub];
  const int ed = E.edofs;
  const int64_t ld = 2 * (int64_t)E.m_pad;
  const double* V = work + E.v_ofs;
  const int* iperm = P.iperm + S.diag0;
  for (int e = blockIdx.x; e < E.nelem; e += gridDim.x) {
    const int* dof = eldofs + E.el_dofs + (int64_t)e * ed;
    const double* dK = eldk + E.el_dk + (int64_t)e * E.dk_stride;
    __syncthreads();
    if (tid < ed) ridx[tid] = iperm[dof[tid]];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};  // entries (a, b) = tid + 256 q
    for (int k0 = 0; k0 < E.m_pad; k0 += kKW) {
      __syncthreads();
      for (int idx = tid; idx < ed * kKW; idx += kAT) {
        const int a = idx / kKW, k = idx % kKW;
        const double* row = V + (int64_t)ridx[a] * ld + k0 + k;
        Zs[a][k] = row[0];
        Ys[a][k] = row[E.m_pad];
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int idx = tid + kAT * q;
        if (idx < ed * ed) {
          const int a = idx / ed, b = idx % ed;
          double sum = 0.0;
#pragma unroll 8
          for (int k = 0; k < kKW; ++k) sum = fma(Ys[b][k], Zs[a][k], sum);
          acc[q] += sum;
        }
      }
    }
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + kAT * q;
      if (idx < ed * ed) t = fma(dK[idx], acc[q], t);
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((tid & 31) == 0) red[tid / 32] = t;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int k = 0; k < kAT / 32; ++k) sum += red[k];
      g[E.el_out + e] = -elsc[E.el_out + e] * sum;
    }
  }
}

// ---------------------------------------------------------------- TRSM-path assembly of F_i
//
// After the backward solve, V_Z row iperm[d] holds row d of Z = K_reg^{-1} B^T (columns in sorted order),
// so F = B Z: F[a][b] = s_a Z[dof_a][b].  One CTA per tile of the batch's subdomains writes the stored
// (lower) part in the tile layout and precision of F.
template <typename TF>
__global__ void __launch_bounds__(kAT) zgather_tiles_kernel(DevPlan P, const AdjBatch* B, const TileDesc* desc,
                                                           const int* tile0, const double* work, TF* F) {
  constexpr int E = (int)sizeof(TF), V = 16 / E;
  const AdjBatch& A = B[blockIdx.y];
  const SubInfo& S = P.sub[A.sub];
  const int* iperm = P.iperm + S.diag0;
  const double* Vz = work + A.v_ofs;
  const int ntile = S.nb * (S.nb + 1) / 2;
  for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
    const TileDesc d = desc[tile0[A.sub] + t];
    const bool diag = (d.flags & kTileDiag) != 0;
    TF* Ft = F + d.f_ofs;
    for (int idx = threadIdx.x; idx < d.rows * kT; idx += kAT) {
      const int r = idx / kT, cc = idx % kT;
      if (diag && cc >= V * ((r + V) / V)) continue;  // not stored
      const int a = d.prow + r, b = d.pcol + cc;
      double v = 0.0;
      if (!(diag && cc > r) && P.qmap[a] >= 0 && P.qmap[b] >= 0)
        v = P.qsign[a] * Vz[(int64_t)iperm[P.qdof[a]] * A.m_pad + (b - S.qcol)];
      Ft[diag ? diag_pos<E>(r, cc) : tile_pos(r, cc)] = (TF)v;
    }
  }
}

// ---------------------------------------------------------------- weighted trace
//
// <W_i, F_i> summed over the stored lower tiles of every F_i: an entry (a, b)
// of sorted columns, a > b, weighs W[ra][rb] + W[rb][ra] (F symmetric), a
// diagonal entry W[ra][ra] (ra = B row of sorted column a).  One CTA per tile
// writes its partial; a single CTA sums the partials in tile order.
template <typename TF>
__global__ void __launch_bounds__(kAT) wtrace_tiles_kernel(const TileDesc* desc, int ntiles, const TF* F,
                                                          const int* qmap, const int* colsub, const int* colperm,
                                                          const SubInfo* sub, const int64_t* woff,
                                                          const double* W, double* part) {
  __shared__ double red[kAT / 32];
  const int tid = threadIdx.x;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const TileDesc d = desc[t];
    const TF* Ft = F + d.f_ofs;
    const bool diag = (d.flags & kTileDiag) != 0;
    const int si = colsub[d.prow];
    const int m = sub[si].m;
    const double* Wi = W + woff[si];
    double acc = 0.0;
    for (int idx = tid; idx < d.rows * kT; idx += kAT) {
      const int r = idx / kT, cc = idx % kT;
      if (diag && cc > r) continue;
      const int a = d.prow + r, b = d.pcol + cc;
      if (qmap[a] < 0 || qmap[b] < 0) continue;
      const double f = (double)Ft[diag ? diag_pos<(int)sizeof(TF)>(r, cc) : tile_pos(r, cc)];
      const int ra = colperm[a], rb = colperm[b];
      const double wgt = (a == b) ? Wi[(int64_t)ra * m + ra] : Wi[(int64_t)ra * m + rb] + Wi[(int64_t)rb * m + ra];
      acc = fma(wgt, f, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid / 32] = acc;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int k = 0; k < kAT / 32; ++k) s += red[k];
      part[d.slot] = s;
    }
  }
}

__global__ void __launch_bounds__(kAT) sum_ordered_kernel(const double* part, int n, double* out) {
  __shared__ double red[kAT];
  double s = 0.0;
  // thread t sums a contiguous stretch, then the stretches are added in order
  const int per = (n + kAT - 1) / kAT;
  for (int i = threadIdx.x * per; i < min(n, (threadIdx.x + 1) * per); ++i) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kAT; ++k) t += red[k];
    *out = t;
  }
}

}  // namespace

void launch_adj_wsort(const AdjBatch* B, int nb, const double* W, const int* colperm, double* work, int max_mpad,
                      cudaStream_t st) {
  if (nb <= 0) return;
  const int64_t tot = (int64_t)max_mpad * max_mpad;
  dim3 grid((unsigned)std::min<int64_t>((tot + kAT - 1) / kAT, 1024), (unsigned)nb);
  wsort_kernel<<<grid, kAT, 0, st>>>(B, nb, W, colperm, work);
}

void launch_adj_build(const DevPlan& P, const AdjBatch* B, const int4* items, int nitems, int* queue,
                      const double* Xu, double* work, int grid, cudaStream_t st) {
  if (nitems > 0) adj_build_kernel<<<grid, kAT, 0, st>>>(P, B, items, nitems, queue, Xu, work);
}

void launch_adj_bsolve(const DevPlan& P, const AdjBatch* B, const int2* items, int nitems, int* queue, double* work,
                       int grid, cudaStream_t st) {
  if (nitems > 0) adj_bsolve_kernel<<<grid, kAT, 0, st>>>(P, B, items, nitems, queue, work);
}

void launch_adj_contract(const DevPlan& P, const AdjBatch* B, int nb, int max_nelem, const int* eldofs,
                         const double* eldk, const double* elsc, const double* work, double* g, cudaStream_t st) {
  if (nb <= 0 || max_nelem <= 0) return;
  dim3 grid((unsigned)std::min(max_nelem, 4096), (unsigned)nb);
  adj_contract_kernel<<<grid, kAT, 0, st>>>(P, B, nb, eldofs, eldk, elsc, work, g);
}

void launch_zgather_tiles(const DevPlan& P, const AdjBatch* B, int nb, const TileDesc* desc, const int* tile0,
                          const double* work, bool fp32, void* F, int max_tiles, cudaStream_t st) {
  if (nb <= 0) return;
  dim3 grid((unsigned)std::max(1, std::min(max_tiles, 1024)), (unsigned)nb);
  if (fp32) zgather_tiles_kernel<float><<<grid, kAT, 0, st>>>(P, B, desc, tile0, work, (float*)F);
  else zgather_tiles_kernel<double><<<grid, kAT, 0, st>>>(P, B, desc, tile0, work, (double*)F);
}

void launch_weighted_trace(bool fp32, const TileDesc* desc, int ntiles, const void* F, const int* qmap,
                           const int* colsub, const int* colperm, const SubInfo* sub, const int64_t* woff,
                           const double* W, double* part, double* out, int grid, cudaStream_t st) {
  if (ntiles > 0) {
    if (fp32)
      wtrace_tiles_kernel<float><<<grid, kAT, 0, st>>>(desc, ntiles, (const float*)F, qmap, colsub, colperm, sub,
                                                       woff, W, part);
    else
      wtrace_tiles_kernel<double><<<grid, kAT, 0, st>>>(desc, ntiles, (const double*)F, qmap, colsub, colperm, sub,
                                                        woff, W, part);
  }
  sum_ordered_kernel<<<1, kAT, 0, st>>>(part, ntiles, out);
}

}  // namespace feti
