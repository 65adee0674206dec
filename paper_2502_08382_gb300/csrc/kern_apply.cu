// Explicit application q = F p (paper eq. 12 summed over subdomains, with
// Algorithm 2's scatter / per-subdomain apply / gather), three launches:
//
//  1. scatter:  pg[j] = p[map_i(j)] for every sorted column j of every
//               subdomain (FP32 for FP32 tiles, FP64 for FP64 tiles);
//  2. tiles:    a persistent kernel streams the lower tiles of all F_i from
//               HBM with 1D bulk copies (cp.async.bulk + mbarrier
//               complete_tx) through a ring of shared-memory stages.  A work
//               item is up to kChunk consecutive tiles (b, bj0..bj1) of one
//               tile row, which are contiguous in memory.  For each tile the
//               CTA forms the row partial F_t p_bj (accumulated over the
//               item) and, off the diagonal, the column partial F_t^T p_b;
//               both go to small per-item / per-tile scratch slots;
//  3. gather:   q[lambda] = sum over the (at most two) subdomain columns of
//               lambda of their row and column partials, in a fixed order
//               (deterministic, no atomics).
// Tile arithmetic runs in the tile's precision (FP32 tiles: FP32 FMAs over
// 64 terms); the cross-tile sums in phase 3 are FP64.
#include "common.cuh"
#include "kernels.h"

namespace feti {
namespace {

constexpr int kApplyThreads = 256;
template <typename TF>
struct ApplyCfg {
  static constexpr int kStages = sizeof(TF) == 4 ? 6 : 3;
};

__device__ __forceinline__ uint32_t smem_u32a(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_test_a(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

template <typename TF>
__global__ void scatter_kernel(const int* qmap, int64_t ncols, const double* p, TF* pg) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ncols; g += (int64_t)gridDim.x * blockDim.x) {
    const int lam = qmap[g];
    pg[g] = lam >= 0 ? (TF)p[lam] : (TF)0;
  }
}

// Cursor over this CTA's flattened tile sequence (items blockIdx.x + k * gridDim.x).
struct TileCursor {
  int item, tile;  // item index into the list, tile offset inside the item
};

template <typename TF>
__global__ void __launch_bounds__(kApplyThreads, 2) apply_tiles_kernel(DevPlan P, const int4* items, int nitems,
                                                                      const TF* F, const TF* pg, TF* rowpart,
                                                                      TF* colpart, int* status) {
  constexpr int kTileBytes = kT * kT * (int)sizeof(TF);
  constexpr int kStagesA = ApplyCfg<TF>::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  __shared__ uint64_t full[kStagesA];
  __shared__ TF prow[kT], pcol[kT];
  __shared__ TF cred[16][kT + 1];
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  const int rg = tid / 16, cg = tid % 16;  // 4 x 4 block: rows 4 rg .. 4 rg + 3, columns 4 cg .. 4 cg + 3
  if (tid == 0) {
    for (int s = 0; s < kStagesA; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32a(&full[s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  __syncthreads();
  // producer state (thread 0 only)
  TileCursor pc{(int)blockIdx.x, 0};
  uint32_t issued = 0;
  auto produce = [&]() {
    // issue the next tile of this CTA's sequence, if any
    while (pc.item < nitems && pc.tile >= items[pc.item].w - items[pc.item].z) {
      pc.item += gridDim.x;
      pc.tile = 0;
    }
    if (pc.item >= nitems) return;
    const int4 it = items[pc.item];
    const SubInfo& S = P.sub[it.x];
    const int b = it.y, bj = it.z + pc.tile;
    const TF* src = F + S.F + (int64_t)(b * (b + 1) / 2 + bj) * kT * kT;
    const int st = issued % kStagesA;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    bulk_load(smem_u32a(smem + st * kTileBytes), src, kTileBytes, smem_u32a(&full[st]));
    ++issued;
    ++pc.tile;
  };
  if (tid == 0)
    for (int s = 0; s < kStagesA; ++s) produce();

  uint32_t consumed = 0;
  for (int ii = blockIdx.x; ii < nitems; ii += gridDim.x) {
    const int4 it = items[ii];
    const SubInfo S = P.sub[it.x];
    const int b = it.y;
    __syncthreads();
    if (tid < kT) prow[tid] = pg[S.qcol + b * kT + tid];
    TF racc[4] = {(TF)0, (TF)0, (TF)0, (TF)0};
    for (int bj = it.z; bj < it.w; ++bj) {
      const int st = consumed % kStagesA;
      if (tid < kT) pcol[tid] = pg[S.qcol + bj * kT + tid];
      if (tid == 0) {
        bool ok = false;
        for (int spin = 0; spin < (1 << 25); ++spin) {
          if (mbar_test_a(smem_u32a(&full[st]), (consumed / kStagesA) & 1)) {
            ok = true;
            break;
          }
          __nanosleep(20);
        }
        if (!ok) s_abort = 1;
      }
      __syncthreads();
      if (s_abort) break;
      const TF* Ft = reinterpret_cast<const TF*>(smem + st * kTileBytes);
      TF v[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const TF* rowp = Ft + (4 * rg + a) * kT + 4 * cg;
#pragma unroll
        for (int c = 0; c < 4; ++c) v[a][c] = rowp[c];
      }
      // row partial: rows 4rg+a over columns 4cg..4cg+3 (reduced over cg after the item)
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        TF s = (TF)0;
#pragma unroll
        for (int c = 0; c < 4; ++c) s = fma(v[a][c], pcol[4 * cg + c], s);
        racc[a] += s;
      }
      if (bj < b) {
        // column partial: columns 4cg+c over rows 4rg..4rg+3, reduced over rg through shared memory
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          TF s = (TF)0;
#pragma unroll
          for (int a = 0; a < 4; ++a) s = fma(v[a][c], prow[4 * rg + a], s);
          cred[rg][4 * cg + c] = s;
        }
      }
      __syncthreads();  // stage fully read; column partials staged
      ++consumed;
      if (tid == 0) produce();
      if (bj < b && tid < kT) {
        TF s = (TF)0;
#pragma unroll
        for (int r = 0; r < 16; ++r) s += cred[r][tid];
        colpart[S.tpart + (int64_t)(b * (b + 1) / 2 + bj) * kT + tid] = s;
      }
    }
    if (s_abort) break;
    // reduce the row partial over the 16 column groups (lanes cg within a half warp)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      TF s = racc[a];
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      racc[a] = s;
    }
    if (cg == 0) {
      const int nch = (S.nb + kApplyChunk - 1) / kApplyChunk;
      const int chunk = it.z / kApplyChunk;
      TF* dst = rowpart + S.rpart + ((int64_t)b * nch + chunk) * kT + 4 * rg;
#pragma unroll
      for (int a = 0; a < 4; ++a) dst[a] = racc[a];
    }
  }
  if (s_abort && tid == 0) atomicOr(status, kStatTimeout);
  // drain: wait (bounded) for copies this CTA issued but did not consume
  if (tid == 0) {
    while (consumed < issued) {
      const int st = consumed % kStagesA;
      bool ok = false;
      for (int spin = 0; spin < (1 << 25); ++spin) {
        if (mbar_test_a(smem_u32a(&full[st]), (consumed / kStagesA) & 1)) {
          ok = true;
          break;
        }
        __nanosleep(20);
      }
      if (!ok) break;
      ++consumed;
    }
  }
  __syncthreads();
}

// q[lambda] = sum over its subdomain columns g of (row partials of g's block
// over the item chunks) + (column partials of the tiles below g's block).
template <typename TF>
__global__ void gather_kernel(DevPlan P, const int* colsub, const int* c0, const int* c1, int nlam,
                              const TF* rowpart, const TF* colpart, double* q) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlam; l += gridDim.x * blockDim.x) {
    double tot = 0.0;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int g = e == 0 ? c0[l] : c1[l];
      if (g < 0) continue;
      const SubInfo& S = P.sub[colsub[g]];
      const int j = (int)(g - S.qcol), b = j / kT, x = j % kT;
      const int nch = (S.nb + kApplyChunk - 1) / kApplyChunk;
      double s = 0.0;
      for (int c = 0; c * kApplyChunk <= b; ++c) s += (double)rowpart[S.rpart + ((int64_t)b * nch + c) * kT + x];
      for (int bi = b + 1; bi < S.nb; ++bi) s += (double)colpart[S.tpart + (int64_t)(bi * (bi + 1) / 2 + b) * kT + x];
      tot += s;
    }
    q[l] = tot;
  }
}

}  // namespace

size_t apply_tiles_smem(bool fp32) {
  return fp32 ? (size_t)ApplyCfg<float>::kStages * kT * kT * 4 + 128 : (size_t)ApplyCfg<double>::kStages * kT * kT * 8 + 128;
}

template <typename TF>
static void launch_apply_t(const DevPlan& P, const int4* items, int nitems, const void* F, const int* qmap,
                           int64_t ncols, const double* p, void* pg, void* rowpart, void* colpart, const int* colsub,
                           const int* c0, const int* c1, int nlam, double* q, int grid, int* status, cudaStream_t st) {
  const int sg = (int)std::min<int64_t>((ncols + 255) / 256, 152 * 8);
  const size_t smem = apply_tiles_smem(sizeof(TF) == 4);
  scatter_kernel<TF><<<std::max(sg, 1), 256, 0, st>>>(qmap, ncols, p, (TF*)pg);
  cudaFuncSetAttribute(apply_tiles_kernel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  apply_tiles_kernel<TF><<<grid, kApplyThreads, smem, st>>>(P, items, nitems, (const TF*)F, (const TF*)pg,
                                                           (TF*)rowpart, (TF*)colpart, status);
  const int gg = std::max(1, std::min((nlam + 255) / 256, 152 * 8));
  gather_kernel<TF><<<gg, 256, 0, st>>>(P, colsub, c0, c1, nlam, (const TF*)rowpart, (const TF*)colpart, q);
}

void launch_apply(const DevPlan& P, bool fp32, const int4* items, int nitems, const void* F, const int* qmap,
                  int64_t ncols, const double* p, void* pg, void* rowpart, void* colpart, const int* colsub,
                  const int* c0, const int* c1, int nlam, double* q, int grid, int* status, cudaStream_t st) {
  if (fp32)
    launch_apply_t<float>(P, items, nitems, F, qmap, ncols, p, pg, rowpart, colpart, colsub, c0, c1, nlam, q, grid,
                          status, st);
  else
    launch_apply_t<double>(P, items, nitems, F, qmap, ncols, p, pg, rowpart, colpart, colsub, c0, c1, nlam, q, grid,
                           status, st);
}

}  // namespace feti
