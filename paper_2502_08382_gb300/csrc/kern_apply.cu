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

#include "../../include/feti.h"
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

template <typename TF>
__global__ void __launch_bounds__(kApplyThreads, 2) apply_tiles_kernel(DevPlan P, const int4* items, int nitems,
                                                                      const TF* F, const TF* pg, TF* rowpart,
                                                                      TF* colpart, int* status) {
  using C = ApplyCfg<TF>;
  constexpr int S = C::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  __shared__ uint64_t full[S], empty[S];
  __shared__ TF cred[S][kConsumerWarps][kT];
  __shared__ int cnt[S];
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
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
    uint32_t t = 0;
    for (int ii = blockIdx.x; ii < nitems && !s_abort; ii += gridDim.x) {
      const int4 it = items[ii];
      const SubInfo& Sb = P.sub[it.x];
      const int b = it.y;
      for (int bj = it.z; bj < it.w; ++bj, ++t) {
        const int st = t % S;
        if (t >= S && !warp_wait(smem_u32a(&empty[st]), ((t / S) + 1) & 1)) {
          s_abort = 1;
          break;
        }
        if (lane == 0) {
          const uint32_t stage = smem_u32a(smem + st * C::kStageBytes);
          const uint32_t fb = smem_u32a(&full[st]);
          const TF* src = F + Sb.F + tile_offset(Sb.nb, Sb.vr, b, bj);
          const uint32_t tb = (uint32_t)tile_rows(Sb.nb, Sb.vr, b) * kT * (uint32_t)sizeof(TF);
          expect_tx(fb, tb + 2 * kT * (uint32_t)sizeof(TF));
          bulk_copy(stage, src, tb, fb);
          bulk_copy(stage + C::kTileBytes, pg + Sb.qcol + b * kT, kT * sizeof(TF), fb);
          bulk_copy(stage + C::kTileBytes + kT * sizeof(TF), pg + Sb.qcol + bj * kT, kT * sizeof(TF), fb);
        }
        __syncwarp();
      }
    }
    // drain: every issued copy must land before the CTA exits
    if (s_abort) {
      for (uint32_t u = (t > S ? t - S : 0); u < t; ++u) warp_wait(smem_u32a(&full[u % S]), (u / S) & 1);
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  const int rg = tid / 16, cg = tid % 16;  // 4 x 4 block: rows 4 rg .. 4 rg + 3, columns 4 cg .. 4 cg + 3
  uint32_t t = 0;
  for (int ii = blockIdx.x; ii < nitems; ii += gridDim.x) {
    const int4 it = items[ii];
    const SubInfo& Sb = P.sub[it.x];
    const int b = it.y;
    TF racc[4] = {(TF)0, (TF)0, (TF)0, (TF)0};
    bool ok = true;
    for (int bj = it.z; bj < it.w; ++bj, ++t) {
      const int st = t % S;
      if (!warp_wait(smem_u32a(&full[st]), (t / S) & 1)) {
        ok = false;
        break;
      }
      const uint8_t* stage = smem + st * C::kStageBytes;
      const TF* Ft = reinterpret_cast<const TF*>(stage);
      const TF* pr = reinterpret_cast<const TF*>(stage + C::kTileBytes);
      const TF* pc = pr + kT;
      // rows at or beyond the tile's stored rows hold stale data: read as zero
      const int nrow = tile_rows(Sb.nb, Sb.vr, b);
      TF v[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const TF* rowp = Ft + (4 * rg + a) * kT + 4 * cg;
        const bool in = 4 * rg + a < nrow;
#pragma unroll
        for (int c = 0; c < 4; ++c) v[a][c] = in ? rowp[c] : (TF)0;
      }
      TF pcv[4], prv[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        pcv[c] = pc[4 * cg + c];
        prv[c] = pr[4 * rg + c];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        TF s = (TF)0;
#pragma unroll
        for (int c = 0; c < 4; ++c) s = fma(v[a][c], pcv[c], s);
        racc[a] += s;
      }
      if (bj < b) {
        TF cs[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          TF s = (TF)0;
#pragma unroll
          for (int a = 0; a < 4; ++a) s = fma(v[a][c], prv[a], s);
          cs[c] = s + __shfl_xor_sync(0xffffffffu, s, 16);  // the warp's two row groups
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
            TF s = (TF)0;
#pragma unroll
            for (int w = 0; w < kConsumerWarps; ++w) s += cred[st][w][c];
            colpart[Sb.tpart + (int64_t)(b * (b + 1) / 2 + bj) * kT + c] = s;  // per-tile slots (unragged)
          }
          if (lane == 0) cnt[st] = 0;
          __syncwarp();
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32a(&empty[st]));
    }
    if (!ok) {
      s_abort = 1;
      break;
    }
    // row partial: reduce over the 16 column groups (lanes of a half warp)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      TF s = racc[a];
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      racc[a] = s;
    }
    if (cg == 0) {
      const int nch = (Sb.nb + kApplyChunk - 1) / kApplyChunk;
      const int chunk = it.z / kApplyChunk;
      TF* dst = rowpart + Sb.rpart + ((int64_t)b * nch + chunk) * kT + 4 * rg;
#pragma unroll
      for (int a = 0; a < 4; ++a) dst[a] = racc[a];
    }
  }
  if (s_abort && tid == 0) atomicOr(status, kStatTimeout);
}

// q_i[j] = (row partials of block b(j) over the item chunks) + (column
// partials of the tiles below block b(j)); one warp per (subdomain, block),
// lanes over the 64 columns of the block.  FP64 sums in a fixed order.
template <typename TF>
__global__ void reduce_cols_kernel(DevPlan P, const int2* blocks, int nblocks, const TF* rowpart,
                                   const TF* colpart, double* qi) {
  const int lane = threadIdx.x & 31;
  for (int wb = (blockIdx.x * blockDim.x + threadIdx.x) / 32; wb < nblocks; wb += gridDim.x * blockDim.x / 32) {
    const int2 sb = blocks[wb];
    const SubInfo& S = P.sub[sb.x];
    const int b = sb.y, nb = S.nb;
    const int nch = (nb + kApplyChunk - 1) / kApplyChunk;
    const int64_t rp = S.rpart, tp = S.tpart, qc = S.qcol;
    for (int x = lane; x < kT; x += 32) {
      double s = 0.0;
      for (int c = 0; c * kApplyChunk <= b; ++c) s += (double)rowpart[rp + ((int64_t)b * nch + c) * kT + x];
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
  return fp32 ? (size_t)ApplyCfg<float>::kStages * ApplyCfg<float>::kStageBytes + 128
              : (size_t)ApplyCfg<double>::kStages * ApplyCfg<double>::kStageBytes + 128;
}

template <typename TF>
static void launch_apply_t(const DevPlan& P, const int4* items, int nitems, const void* F, const int* qmap,
                           int64_t ncols, const double* p, void* pg, void* rowpart, void* colpart, const int2* blocks,
                           int nblocks, double* qi, const int* c0, const int* c1, int nlam, double* q, int grid,
                           int* status, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  const int sg = (int)std::max<int64_t>(1, std::min<int64_t>((ncols + 255) / 256, 152 * 8));
  scatter_kernel<TF><<<sg, 256, 0, st>>>(qmap, ncols, p, (TF*)pg);
  const size_t smem = apply_tiles_smem(sizeof(TF) == 4);
  cudaFuncSetAttribute(apply_tiles_kernel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e0) cudaEventRecord(e0, st);
  apply_tiles_kernel<TF><<<grid, kApplyThreads, smem, st>>>(P, items, nitems, (const TF*)F, (const TF*)pg,
                                                           (TF*)rowpart, (TF*)colpart, status);
  if (e1) cudaEventRecord(e1, st);
  const int rg = std::max(1, std::min((nblocks + 7) / 8, 152 * 16));
  reduce_cols_kernel<TF><<<rg, 256, 0, st>>>(P, blocks, nblocks, (const TF*)rowpart, (const TF*)colpart, qi);
  const int gg = std::max(1, std::min((nlam + 255) / 256, 152 * 8));
  gather_lambda_kernel<<<gg, 256, 0, st>>>(c0, c1, nlam, qi, q);
}

void launch_gather_lambda(const int* c0, const int* c1, int nlam, const double* qi, double* q, cudaStream_t st) {
  const int gg = std::max(1, std::min((nlam + 255) / 256, 152 * 8));
  gather_lambda_kernel<<<gg, 256, 0, st>>>(c0, c1, nlam, qi, q);
}

void launch_apply(const DevPlan& P, bool fp32, const int4* items, int nitems, const void* F, const int* qmap,
                  int64_t ncols, const double* p, void* pg, void* rowpart, void* colpart, const int2* blocks,
                  int nblocks, double* qi, const int* c0, const int* c1, int nlam, double* q, int grid, int* status,
                  cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  if (fp32)
    launch_apply_t<float>(P, items, nitems, F, qmap, ncols, p, pg, rowpart, colpart, blocks, nblocks, qi, c0, c1,
                          nlam, q, grid, status, st, e0, e1);
  else
    launch_apply_t<double>(P, items, nitems, F, qmap, ncols, p, pg, rowpart, colpart, blocks, nblocks, qi, c0, c1,
                           nlam, q, grid, status, st, e0, e1);
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
constexpr int kStaticMaxItems = kStaticMaxNb * ((kStaticMaxNb + kApplyChunk - 1) / kApplyChunk);

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];
static __device__ __align__(256) int4 g_static_items[kStaticMaxItems];
static __device__ __align__(256) int2 g_static_blocks[kStaticMaxNb];
static __device__ __align__(256) SubInfo g_static_sub;
static __device__ __align__(256) int g_static_status;

namespace {

// Describe the single subdomain, its work items and blocks in the static
// arrays, zero the padding of the gathered p, and clear the status word
// (the only state that must start at zero; every other slot is overwritten).
template <typename TF>
__global__ void static_setup_kernel(int m, int nb, int64_t rpart, int64_t tpart, TF* pg) {
  if (threadIdx.x == 0) {
    SubInfo S{};
    S.m = m;
    S.m_pad = nb * kT;
    S.nb = nb;
    S.vr = m - kT * (nb - 1);
    S.F = 0;
    S.qcol = 0;
    S.rpart = rpart;
    S.tpart = tpart;
    g_static_sub = S;
    g_static_status = 0;
    int k = 0;
    for (int b = 0; b < nb; ++b)
      for (int c = 0; c <= b; c += kApplyChunk) g_static_items[k++] = make_int4(0, b, c, min(c + kApplyChunk, b + 1));
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
  int4* items = nullptr;
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
    if ((e = cudaGetSymbolAddress((void**)&a.items, g_static_items)) != cudaSuccess) return e;
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
  // scratch layout: [pg: m_pad TF][row partials: nb nch kT TF][column partials: ntile kT TF] | [qi: m_pad double]
  const int64_t n_pg = m_pad, n_row = (int64_t)nb * nch * kT, n_col = ntile * kT;
  const int64_t qi_ofs = ((n_pg + n_row + n_col) * (int64_t)sizeof(TF) + 255) / 256 * 256 / 8;
  if (qi_ofs + m_pad > kStaticDoubles || nitems > kStaticMaxItems) return FETI_ERR_ARG;
  StaticAddrs a;
  if (static_addresses(a) != cudaSuccess) return FETI_ERR_CUDA;
  TF* pg = reinterpret_cast<TF*>(a.scratch);
  double* qi = a.scratch + qi_ofs;
  static_setup_kernel<TF><<<1, 256, 0, st>>>(m, nb, n_pg, n_pg + n_row, pg);
  scatter_kernel<TF><<<std::max(1, (m + 255) / 256), 256, 0, st>>>(map, m, p, pg);
  DevPlan P{};
  P.sub = a.sub;
  // row / column partial slots are the offsets S.rpart / S.tpart from the scratch base
  const size_t smem = apply_tiles_smem(sizeof(TF) == 4);
  cudaFuncSetAttribute(apply_tiles_kernel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int grid = std::max(1, std::min(nitems, 152 * 2));
  apply_tiles_kernel<TF><<<grid, kApplyThreads, smem, st>>>(P, a.items, nitems, F, pg, pg, pg, a.status);
  reduce_cols_kernel<TF><<<std::max(1, (nb + 7) / 8), 256, 0, st>>>(P, a.blocks, nb, pg, pg, qi);
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
