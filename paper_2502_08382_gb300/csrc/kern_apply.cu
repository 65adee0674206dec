// Explicit application q = F p (paper eq. 12 summed over subdomains, with
// Algorithm 2's scatter / per-subdomain apply / gather), three launches:
//
//  0. scatter: pg[j] = p[map_i(j)] for every sorted column j of every
//             subdomain (Algorithm 2's scatter), in the tile precision;
//  1. tiles:  a persistent, warp-specialised kernel streams the lower tiles
//             of all F_i from HBM.  Lane 0 of warp 8 is the producer: for each
//             tile it issues 1D bulk copies (cp.async.bulk + mbarrier
//             complete_tx) of the contiguous 16 KB (FP32) / 32 KB (FP64) tile
//             and of the two 64-entry segments of pg it needs into a ring of
//             shared-memory stages.  Warps 0-7 consume: per tile the row partial F_t p_bj
//             (accumulated over the work item) and, off the diagonal, the
//             column partial F_t^T p_b.  A work item is up to kApplyChunk
//             consecutive tiles (b, bj0..bj1) of one tile row (contiguous in
//             memory).  Stages are released through per-stage `empty`
//             mbarriers; the last consumer warp to finish a tile sums the 8
//             per-warp column partials (no CTA-wide barrier in the loop).
//  2. gather: q[lambda] = sum over the (at most two) subdomain columns of
//             lambda of their row and column partials, in a fixed order
//             (deterministic, no atomics on values).
// Tile arithmetic runs in the tile's precision (FP32 tiles: FP32 FMAs over
// 64 terms); the cross-tile sums in phase 2 are FP64.  All waits are bounded.
#include <mutex>

#include "feti.h"
#include "common.cuh"
#include "kernels.h"

namespace feti {
namespace {

constexpr int kConsumerWarps = 8;
constexpr int kApplyThreads = (kConsumerWarps + 1) * 32;
template <typename TF>
struct ApplyCfg {
  static constexpr int kStages = sizeof(TF) == 4 ? 5 : 2;
  static constexpr int kTileBytes = kT * kT * (int)sizeof(TF);
  static constexpr int kStageBytes = kTileBytes + 2 * kT * (int)sizeof(TF);
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

__device__ __forceinline__ bool mbar_try_a(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// lane 0 waits (try_wait, bounded by about 2e9 clock cycles), result broadcast to the warp
__device__ __forceinline__ bool warp_wait(uint32_t mbar, uint32_t parity) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) {
    const long long t0 = clock64();
    while (!(ok = mbar_try_a(mbar, parity))) {
      if (clock64() - t0 > 2000000000LL) break;
    }
  }
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
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

// One stage: the tile, the two p segments it needs, and its descriptor.
// NS = number of stages in the ring (the autotuner picks it per problem).
template <typename TF, int NS>
__global__ void __launch_bounds__(kApplyThreads) apply_tiles_kernel(const TileDesc* desc, const int* cta_begin,
                                                                   const TF* F, const TF* pg, TF* rowpart,
                                                                   TF* colpart, int* status) {
  using C = ApplyCfg<TF>;
  constexpr int S = NS;
  constexpr int kMeta = 64;  // bytes of descriptor kept after the p segments
  constexpr int kStride = C::kStageBytes + kMeta;
  constexpr int cw = 16 / (int)sizeof(TF), nchk = kT / cw;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  __shared__ uint64_t full[S], empty[S];
  __shared__ TF cred[S][kConsumerWarps][kT];
  __shared__ int cnt[S];
  __shared__ TileDesc dring[64];
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int t0 = cta_begin[blockIdx.x], t1 = cta_begin[blockIdx.x + 1];
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32a(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32a(&empty[s])), "r"(kConsumerWarps));
      cnt[s] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  __syncthreads();

  if (warp == kConsumerWarps) {
    // ------------------------------------------------------------ producer
    uint32_t k = 0;
    for (int t = t0; t < t1 && !s_abort; ++t, ++k) {
      if (((t - t0) & 31) == 0) {
        // prefetch the next 32 descriptors into a double-buffered ring
        const int base = ((t - t0) >> 5) & 1;
        if (t + lane < t1) dring[base * 32 + lane] = desc[t + lane];
        __syncwarp();
      }
      const TileDesc d = dring[(((t - t0) >> 5) & 1) * 32 + ((t - t0) & 31)];
      const int st = k % S;
      if (k >= S && !warp_wait(smem_u32a(&empty[st]), ((k / S) + 1) & 1)) {
        s_abort = 1;
        break;
      }
      if (lane == 0) {
        uint8_t* stage = smem + st * kStride;
        *reinterpret_cast<TileDesc*>(stage + C::kStageBytes) = d;
        const uint32_t sa = smem_u32a(stage);
        const uint32_t fb = smem_u32a(&full[st]);
        const uint32_t tb = (uint32_t)d.rows * kT * (uint32_t)sizeof(TF);
        expect_tx(fb, tb + 2 * kT * (uint32_t)sizeof(TF));
        bulk_copy(sa, F + d.f_ofs, tb, fb);
        bulk_copy(sa + C::kTileBytes, pg + d.prow, kT * sizeof(TF), fb);
        bulk_copy(sa + C::kTileBytes + kT * sizeof(TF), pg + d.pcol, kT * sizeof(TF), fb);
      }
      __syncwarp();
    }
    if (s_abort) {
      for (uint32_t u = (k > S ? k - S : 0); u < k; ++u) warp_wait(smem_u32a(&full[u % S]), (u / S) & 1);
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  // thread (rg, cg) holds the 4 x 4 block rows 4 rg .. 4 rg + 3, columns
  // 4 cg .. 4 cg + 3 (one 16-byte chunk per row for FP32, two for FP64);
  // the stored rows are chunk-swizzled (tile_pos), which keeps the reads of a
  // quarter warp on distinct banks.  The column partial of an off-diagonal
  // tile is summed over the 8 warps by the last warp to finish it.
  const int rg = tid / 16, cg = tid % 16;
  TF racc[4] = {(TF)0, (TF)0, (TF)0, (TF)0};
  uint32_t k = 0;
  for (int t = t0; t < t1; ++t, ++k) {
    const int st = k % S;
    if (!warp_wait(smem_u32a(&full[st]), (k / S) & 1)) {
      s_abort = 1;
      break;
    }
    const uint8_t* stage = smem + st * kStride;
    const TileDesc d = *reinterpret_cast<const TileDesc*>(stage + C::kStageBytes);
    const TF* Ft = reinterpret_cast<const TF*>(stage);
    const TF* pr = reinterpret_cast<const TF*>(stage + C::kTileBytes);
    const TF* pc = pr + kT;
    TF v[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = 4 * rg + a;
      const bool in = r < d.rows;  // rows beyond the stored ones hold stale data: read as zero
      if constexpr (sizeof(TF) == 4) {
        const float4 x = *reinterpret_cast<const float4*>(Ft + r * kT + ((cg ^ (r % nchk)) * cw));
        v[a][0] = in ? x.x : 0.f;
        v[a][1] = in ? x.y : 0.f;
        v[a][2] = in ? x.z : 0.f;
        v[a][3] = in ? x.w : 0.f;
      } else {
        const double2 x0 = *reinterpret_cast<const double2*>(Ft + r * kT + (((2 * cg) ^ (r % nchk)) * cw));
        const double2 x1 = *reinterpret_cast<const double2*>(Ft + r * kT + (((2 * cg + 1) ^ (r % nchk)) * cw));
        v[a][0] = in ? x0.x : 0.0;
        v[a][1] = in ? x0.y : 0.0;
        v[a][2] = in ? x1.x : 0.0;
        v[a][3] = in ? x1.y : 0.0;
      }
    }
    TF pcv[4], prv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      pcv[c] = pc[4 * cg + c];
      prv[c] = pr[4 * rg + c];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      TF s2 = (TF)0;
#pragma unroll
      for (int c = 0; c < 4; ++c) s2 = fma(v[a][c], pcv[c], s2);
      racc[a] += s2;
    }
    if (d.col_slot >= 0) {
      TF cs[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        TF s2 = (TF)0;
#pragma unroll
        for (int a = 0; a < 4; ++a) s2 = fma(v[a][c], prv[a], s2);
        cs[c] = s2 + __shfl_xor_sync(0xffffffffu, s2, 16);  // the warp's two row groups
      }
      if (lane < 16) {
#pragma unroll
        for (int c = 0; c < 4; ++c) cred[st][warp][4 * cg + c] = cs[c];
      }
      __syncwarp();
      int last = 0;
      if (lane == 0) {
        __threadfence_block();
        last = atomicAdd(&cnt[st], 1) == kConsumerWarps - 1;
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      if (last) {
        __threadfence_block();
        for (int c = lane; c < kT; c += 32) {
          TF s2 = (TF)0;
#pragma unroll
          for (int w = 0; w < kConsumerWarps; ++w) s2 += cred[st][w][c];
          colpart[(int64_t)d.col_slot * kT + c] = s2;
        }
        if (lane == 0) cnt[st] = 0;
        __syncwarp();
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32a(&empty[st]));
    if (d.flags & kTileLast) {
      // row partial of the work item: reduce over the 16 column groups (lanes of a half warp)
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        TF s2 = racc[a];
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        racc[a] = (TF)0;
        if (cg == 0) rowpart[(int64_t)d.row_slot * kApplyWarps * kT + 4 * rg + a] = s2;
      }
    }
  }
  if (s_abort && tid == 0) atomicOr(status, kStatTimeout);
}

template <typename TF>
size_t stage_smem(int ns) {
  return (size_t)ns * (ApplyCfg<TF>::kStageBytes + 64) + 128;
}

// launch the staged kernel with ns stages (2..6)
template <typename TF>
void launch_tiles(int ns, int grid, cudaStream_t st, const TileDesc* desc, const int* cta_begin, const TF* F,
                  const TF* pg, TF* rowpart, TF* colpart, int* status) {
  const size_t smem = stage_smem<TF>(ns);
#define FETI_TL(N)                                                                                                  \
  case N:                                                                                                           \
    cudaFuncSetAttribute(apply_tiles_kernel<TF, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
    apply_tiles_kernel<TF, N><<<grid, kApplyThreads, smem, st>>>(desc, cta_begin, F, pg, rowpart, colpart, status); \
    break;
  switch (ns) {
    FETI_TL(2) FETI_TL(3) FETI_TL(4) FETI_TL(5) FETI_TL(6)
    default:
      break;
  }
#undef FETI_TL
}

// q_i[j] = (row partials of block b(j) over the item chunks) + (column
// partials of the tiles below block b(j)); one warp per (subdomain, block),
// lanes over the 64 columns of the block.  FP64 sums in a fixed order.
template <typename TF>
__global__ void reduce_cols_kernel(DevPlan P, const int2* blocks, int nblocks, const TF* rowpart,
                                   const TF* colpart, double* qi, int nslots) {
  const int lane = threadIdx.x & 31;
  for (int wb = (blockIdx.x * blockDim.x + threadIdx.x) / 32; wb < nblocks; wb += gridDim.x * blockDim.x / 32) {
    const int2 sb = blocks[wb];
    const SubInfo& S = P.sub[sb.x];
    const int b = sb.y, nb = S.nb;
    const int nch = (nb + kApplyChunk - 1) / kApplyChunk;
    const int64_t rp = S.rpart, tp = S.tpart, qc = S.qcol;
    for (int x = lane; x < kT; x += 32) {
      double s = 0.0;
      for (int c = 0; c * kApplyChunk <= b; ++c)
        for (int w = 0; w < nslots; ++w)
          s += (double)rowpart[rp + (((int64_t)b * nch + c) * kApplyWarps + w) * kT + x];
      for (int bi = b + 1; bi < nb; ++bi) s += (double)colpart[tp + (int64_t)(bi * (bi + 1) / 2 + b) * kT + x];
      qi[qc + b * kT + x] = s;
    }
  }
}

// q[lambda] = its (at most two) subdomain contributions, in subdomain order
__global__ void gather_lambda_kernel(const int* c0, const int* c1, int nlam, const double* qi, double* q) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlam; l += gridDim.x * blockDim.x) {
    const int a = c0[l], b = c1[l];
    double s = a >= 0 ? qi[a] : 0.0;
    if (b >= 0) s += qi[b];
    q[l] = s;
  }
}

}  // namespace

size_t apply_tiles_smem(bool fp32) {
  return fp32 ? stage_smem<float>(ApplyCfg<float>::kStages) : stage_smem<double>(ApplyCfg<double>::kStages);
}

template <typename TF>
static void launch_apply_t(const DevPlan& P, const TileDesc* desc, const int* cta_begin, const void* F,
                           const int* qmap, int64_t ncols, const double* p, void* pg, void* rowpart, void* colpart,
                           const int2* blocks, int nblocks, double* qi, const int* c0, const int* c1, int nlam,
                           double* q, int grid, int* status, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                           int stages) {
  const int sg = (int)std::max<int64_t>(1, std::min<int64_t>((ncols + 255) / 256, 152 * 8));
  scatter_kernel<TF><<<sg, 256, 0, st>>>(qmap, ncols, p, (TF*)pg);
  if (e0) cudaEventRecord(e0, st);
  launch_tiles<TF>(stages, grid, st, desc, cta_begin, (const TF*)F, (const TF*)pg, (TF*)rowpart, (TF*)colpart, status);
  if (e1) cudaEventRecord(e1, st);
  const int rg = std::max(1, std::min((nblocks + 7) / 8, 152 * 16));
  reduce_cols_kernel<TF><<<rg, 256, 0, st>>>(P, blocks, nblocks, (const TF*)rowpart, (const TF*)colpart, qi, 1);
  const int gg = std::max(1, std::min((nlam + 255) / 256, 152 * 8));
  gather_lambda_kernel<<<gg, 256, 0, st>>>(c0, c1, nlam, qi, q);
}

void launch_gather_lambda(const int* c0, const int* c1, int nlam, const double* qi, double* q, cudaStream_t st) {
  const int gg = std::max(1, std::min((nlam + 255) / 256, 152 * 8));
  gather_lambda_kernel<<<gg, 256, 0, st>>>(c0, c1, nlam, qi, q);
}

void launch_apply(const DevPlan& P, bool fp32, const TileDesc* desc, const int* cta_begin, const void* F,
                  const int* qmap, int64_t ncols, const double* p, void* pg, void* rowpart, void* colpart,
                  const int2* blocks, int nblocks, double* qi, const int* c0, const int* c1, int nlam, double* q,
                  int grid, int* status, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int stages) {
  if (fp32)
    launch_apply_t<float>(P, desc, cta_begin, F, qmap, ncols, p, pg, rowpart, colpart, blocks, nblocks, qi, c0, c1,
                          nlam, q, grid, status, st, e0, e1, stages);
  else
    launch_apply_t<double>(P, desc, cta_begin, F, qmap, ncols, p, pg, rowpart, colpart, blocks, nblocks, qi, c0, c1,
                           nlam, q, grid, status, st, e0, e1, stages);
}

int apply_max_ctas_per_sm(bool fp32, int stages) {
  int nb = 0;
  if (fp32) {
    const size_t smem = stage_smem<float>(stages);
#define FETI_OCC(N)                                                                                      if (stages == N) {                                                                                       cudaFuncSetAttribute(apply_tiles_kernel<float, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, apply_tiles_kernel<float, N>, kApplyThreads, smem);    }
    FETI_OCC(2) FETI_OCC(3) FETI_OCC(4) FETI_OCC(5) FETI_OCC(6)
#undef FETI_OCC
  } else {
    const size_t smem = stage_smem<double>(stages);
#define FETI_OCC(N)                                                                                       if (stages == N) {                                                                                        cudaFuncSetAttribute(apply_tiles_kernel<double, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, apply_tiles_kernel<double, N>, kApplyThreads, smem);    }
    FETI_OCC(2) FETI_OCC(3) FETI_OCC(4) FETI_OCC(5) FETI_OCC(6)
#undef FETI_OCC
  }
  return nb;
}

// ---------------------------------------------------------------------------
// Stand-alone application of one local operator without any device allocation.
//
// Some callers cannot allocate device memory when they apply an operator: a
// host framework that has reserved all device memory for its own pool and
// forbids other allocations, or a latency-critical loop in which cudaMalloc
// (which synchronises the device) is not acceptable.  feti_apply_one_static
// serves them: the caller passes F_i, the multiplier map and the dual vectors;
// every intermediate the apply kernels need lives in the fixed device arrays
// below, which exist once per GPU that loads this library and stay resident
// until the process exits.  All calls share these arrays and they keep the
// last call's contents, so calls that overlap on the GPU (other streams,
// other host threads) race; the caller must order them.

constexpr int kStaticMaxM = 8192;                 // largest m accepted
constexpr int kStaticMaxNb = kStaticMaxM / kT;
constexpr int64_t kStaticDoubles = 1 << 20;       // 8 MiB of scratch
constexpr int kStaticMaxTiles = kStaticMaxNb * (kStaticMaxNb + 1) / 2;
constexpr int kStaticGrid = 152 * 2;

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];
static __device__ __align__(256) TileDesc g_static_desc[kStaticMaxTiles];
static __device__ __align__(256) int g_static_cta[kStaticGrid + 1];
static __device__ __align__(256) int2 g_static_blocks[kStaticMaxNb];
static __device__ __align__(256) SubInfo g_static_sub;
static __device__ __align__(256) int g_static_status;

namespace {

// Describe the single subdomain, its tile descriptors, CTA ranges and blocks
// in the static arrays, zero the padding of the gathered p, and clear the
// status word (the only state that must start at zero; every other slot is
// overwritten).
template <typename TF>
__global__ void static_setup_kernel(int m, int nb, int64_t rpart, int64_t tpart, int grid, TF* pg) {
  const int nch = (nb + kApplyChunk - 1) / kApplyChunk;
  const int vr = m - kT * (nb - 1);
  if (threadIdx.x == 0) {
    SubInfo S{};
    S.m = m;
    S.m_pad = nb * kT;
    S.nb = nb;
    S.vr = vr;
    S.rpart = rpart;
    S.tpart = tpart;
    g_static_sub = S;
    g_static_status = 0;
    const int ntile = nb * (nb + 1) / 2;
    int k = 0, cta = 1;
    g_static_cta[0] = 0;
    for (int b = 0; b < nb; ++b)
      for (int c = 0; c * kApplyChunk <= b; ++c) {
        const int bj0 = c * kApplyChunk, bj1 = min(bj0 + kApplyChunk, b + 1);
        for (int bj = bj0; bj < bj1; ++bj) {
          TileDesc d;
          d.f_ofs = tile_offset(nb, vr, b, bj);
          d.rows = tile_rows(nb, vr, b);
          d.flags = (bj == bj0 ? kTileFirst : 0) | (bj == bj1 - 1 ? kTileLast : 0);
          d.prow = b * kT;
          d.pcol = bj * kT;
          d.col_slot = bj < b ? (int)(tpart / kT) + b * (b + 1) / 2 + bj : -1;
          d.row_slot = (int)(rpart / (kT * kApplyWarps)) + b * nch + c;
          g_static_desc[k++] = d;
        }
        if (cta < grid && (double)k >= (double)ntile * cta / grid) g_static_cta[cta++] = k;
      }
    for (; cta <= grid; ++cta) g_static_cta[cta] = k;
  }
  for (int b = threadIdx.x; b < nb; b += blockDim.x) g_static_blocks[b] = make_int2(0, b);
  for (int j = m + threadIdx.x; j < nb * kT; j += blockDim.x) pg[j] = (TF)0;
}

// q[map[j]] += qi[j] for the m real columns (the map holds distinct multipliers)
__global__ void static_accumulate_kernel(const int* map, int m, const double* qi, double* q) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) q[map[j]] += qi[j];
}

struct StaticAddrs {
  double* scratch = nullptr;
  TileDesc* desc = nullptr;
  int* cta = nullptr;
  int2* blocks = nullptr;
  SubInfo* sub = nullptr;
  int* status = nullptr;
};

std::mutex g_static_mu;
StaticAddrs g_static_addr[64];
bool g_static_ready[64] = {};

// Device addresses of the static arrays on the current device.  In host code
// the array names are host-side stand-ins, so the addresses are looked up
// once per device (with that device current) and cached.
cudaError_t static_addresses(StaticAddrs& out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ready[dev]) {
    StaticAddrs a;
    if ((e = cudaGetSymbolAddress((void**)&a.scratch, g_static_scratch)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&a.desc, g_static_desc)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&a.cta, g_static_cta)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&a.blocks, g_static_blocks)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&a.sub, g_static_sub)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&a.status, g_static_status)) != cudaSuccess) return e;
    g_static_addr[dev] = a;
    g_static_ready[dev] = true;
  }
  out = g_static_addr[dev];
  return cudaSuccess;
}

template <typename TF>
feti_status apply_one_static_t(int m, const TF* F, const int* map, const double* p, double* q, cudaStream_t st) {
  const int nb = (m + kT - 1) / kT;
  const int m_pad = nb * kT;
  const int nch = (nb + kApplyChunk - 1) / kApplyChunk;
  const int64_t ntile = (int64_t)nb * (nb + 1) / 2;
  int nitems = 0;
  for (int b = 0; b < nb; ++b) nitems += b / kApplyChunk + 1;
  const int grid = std::max(1, std::min(nitems, kStaticGrid));
  // scratch layout: [pg: m_pad TF, padded][row partials: nb nch kApplyWarps kT TF][column partials: ntile kT TF]
  //                 | [qi: m_pad double]
  const int64_t n_pg = ((int64_t)m_pad + kT * kApplyWarps - 1) / (kT * kApplyWarps) * (kT * kApplyWarps);
  const int64_t n_row = (int64_t)nb * nch * kT * kApplyWarps, n_col = ntile * kT;
  const int64_t qi_ofs = ((n_pg + n_row + n_col) * (int64_t)sizeof(TF) + 255) / 256 * 256 / 8;
  if (qi_ofs + m_pad > kStaticDoubles || ntile > kStaticMaxTiles) return FETI_ERR_ARG;
  StaticAddrs a;
  if (static_addresses(a) != cudaSuccess) return FETI_ERR_CUDA;
  TF* pg = reinterpret_cast<TF*>(a.scratch);
  double* qi = a.scratch + qi_ofs;
  static_setup_kernel<TF><<<1, 256, 0, st>>>(m, nb, n_pg, n_pg + n_row, grid, pg);
  scatter_kernel<TF><<<std::max(1, (m + 255) / 256), 256, 0, st>>>(map, m, p, pg);
  DevPlan P{};
  P.sub = a.sub;
  // row / column partial slots are offsets from the scratch base (S.rpart / S.tpart)
  launch_tiles<TF>(ApplyCfg<TF>::kStages, grid, st, a.desc, a.cta, F, pg, pg, pg, a.status);
  reduce_cols_kernel<TF><<<std::max(1, (nb + 7) / 8), 256, 0, st>>>(P, a.blocks, nb, pg, pg, qi, 1);
  static_accumulate_kernel<<<std::max(1, (m + 255) / 256), 256, 0, st>>>(map, m, qi, q);
  if (cudaGetLastError() != cudaSuccess) return FETI_ERR_CUDA;
  int status = 0;
  if (cudaMemcpyAsync(&status, a.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return FETI_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FETI_ERR_CUDA;
  return (status & kStatTimeout) ? FETI_ERR_TIMEOUT : FETI_OK;
}

}  // namespace
}  // namespace feti

extern "C" feti_status feti_apply_one_static(int32_t m, int32_t fp32, const void* F_dev, const int32_t* map_dev,
                                             const double* p_dev, double* q_dev, void* stream) {
  if (m <= 0 || m > feti::kStaticMaxM || !F_dev || !map_dev || !p_dev || !q_dev) return FETI_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  return fp32 ? feti::apply_one_static_t<float>(m, (const float*)F_dev, map_dev, p_dev, q_dev, st)
              : feti::apply_one_static_t<double>(m, (const double*)F_dev, map_dev, p_dev, q_dev, st);
}
