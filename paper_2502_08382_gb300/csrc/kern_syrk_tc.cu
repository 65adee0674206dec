// Tensor-core SYRK F_i = X_i^T X_i (paper Sec. IV, SYRK path) on sm_103a.
//
// One CTA computes one 128 x 128 tile (BI, BJ), BJ <= BI, of F_i in sorted
// column order:  F[a][b] = sum_s sum_k X_s[a][k] X_s[b][k]  over the supernodes
// s whose column range J_s meets both 128-blocks (pruning: other supernodes
// hold zeros there).  X_s is stored column-major per supernode (column j of
// X holds the w_s values of rows in s, padded to wp), which is the K-major
// operand layout of tcgen05.mma: A = rows a of the tile, B = rows b, K = the
// supernode rows.
//
// Staging: 16-byte cp.async (zero-filled outside J_s and beyond w_s) writes
// each 128 x 32 FP32 chunk (TF32) or 128 x 64 bf16 chunk (split bf16, from the
// hi/lo copy of X the TRSM writes) into the canonical 128-byte-swizzled
// K-major layout (8-row atoms of 1024 B).  One thread issues tcgen05.mma kind::tf32
// (M = N = 128, K = 8) into a 128-column TMEM accumulator and commits to a
// per-stage mbarrier, which releases the stage for the next cp.async.  The
// epilogue reads TMEM with tcgen05.ld 32x32b and writes the 64 x 64 storage
// tiles of the lower triangle.  SPLIT = 1 stages the bf16 hi/lo halves of each
// FP32 value and accumulates hi*hi + hi*lo + lo*hi (kind::f16 with bf16).
// All waits are bounded; on timeout the kernel flags kStatTimeout, drains its
// copies, frees TMEM and returns.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace feti {
namespace {

constexpr int kM = 128;
constexpr int kStages = 3;
constexpr int kTcThreads = 256;
constexpr int kMetaCap = 512;  // contributions per tile whose metadata is staged in shared memory

// what the loader needs of one contributing supernode block
struct Meta {
  long long xofs;  // X offset of the block (elements, relative to the subdomain's X)
  int wp, w, jb, J;
};
constexpr uint32_t kTmemCols = 128;

__device__ __forceinline__ void tile2_of(int t, int& bi, int& bj) {
  int b = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((b + 1) * (b + 2) / 2 <= t) ++b;
  while (b * (b + 1) / 2 > t) --b;
  bi = b;
  bj = t - b * (b + 1) / 2;
}

// Loader cursor over the (supernode, k-chunk) sequence of one tile.
struct Cursor {
  int c, k0;
};

// bytes of one operand buffer (128 rows x 128 B)
constexpr int kOpBytes = kM * 128;

// SPLIT: 0 = TF32; 1 = split bf16, 64-deep chunks in the 128-byte swizzle (one CTA per SM); 2 = split bf16,
// 32-deep chunks in the 64-byte swizzle (half the stage, two CTAs per SM; the same MMAs in the same order)
template <int SPLIT>
struct Cfg {
  static constexpr int kKC = SPLIT == 1 ? 64 : 32;       // K values per chunk (one swizzled row)
  static constexpr int kOps = SPLIT ? 4 : 2;             // A(hi,lo), B(hi,lo) or A, B
  static constexpr int kRowBytes = SPLIT == 2 ? 64 : 128;
  static constexpr int kOp = kM * kRowBytes;             // bytes of one operand part
  static constexpr int kStageBytes = kOps * kOp;
};

// Stage the chunk (supernode s, rows k0..k0+KC) of the A rows (tile block BI)
// and B rows (tile block BJ).  TF32: from the FP32 X block Xs.  Split bf16:
// from the pre-split copy X2 (per column: wp bf16 hi values, then wp lo
// values), so every 16-byte chunk of the swizzled layout is one cp.async;
// on a diagonal tile (BI = BJ) B equals A and only A is staged.
template <int SPLIT>
__device__ __forceinline__ void load_chunk(uint8_t* stage, const float* Xs, const uint16_t* X2s, int wp, int w, int J,
                                           int ca, int cb, int k0, const void* safe, bool diag) {
  const int tid = threadIdx.x;
  if constexpr (!SPLIT) {
    const uint32_t sA = smem_u32(stage), sB = sA + kOpBytes;
    // 2 operands x 128 rows x 8 chunks of 16 B
    for (int idx = tid; idx < 2 * kM * 8; idx += kTcThreads) {
      const int op = idx / (kM * 8), rem = idx % (kM * 8);
      const int m = rem / 8, c = rem % 8;
      const int x = (op ? cb : ca) + m;
      const int k = k0 + 4 * c;
      const bool ok = x >= 0 && x < J && k < w;
      const void* src = ok ? (const void*)(Xs + (int64_t)x * wp + k) : safe;
      const uint32_t dst = (op ? sB : sA) + (m >> 3) * 1024 + (m & 7) * 128 + ((c ^ (m & 7)) << 4);
      cp_async16(dst, src, ok);
    }
  } else if constexpr (SPLIT == 1) {
    // parts: 0 A hi, 1 A lo, 2 B hi, 3 B lo; 64 K values (8 chunks of 8 bf16) per 128-byte row
    const uint32_t s0 = smem_u32(stage);
    const int nparts = diag ? 2 : 4;
    for (int idx = tid; idx < nparts * kM * 8; idx += kTcThreads) {
      const int part = idx / (kM * 8), rem = idx % (kM * 8);
      const int m = rem / 8, c = rem % 8;
      const int x = (part < 2 ? ca : cb) + m;
      const int k = k0 + 8 * c;
      const bool ok = x >= 0 && x < J && k < w;
      const void* src = ok ? (const void*)(X2s + 2 * (int64_t)x * wp + ((part & 1) ? wp : 0) + k) : safe;
      const uint32_t dst = s0 + part * kOpBytes + (m >> 3) * 1024 + (m & 7) * 128 + ((c ^ (m & 7)) << 4);
      cp_async16(dst, src, ok);
    }
  } else {
    // the same parts with 32 K values (4 chunks of 8 bf16) per 64-byte row, 64-byte swizzle
    const uint32_t s0 = smem_u32(stage);
    const int nparts = diag ? 2 : 4;
    for (int idx = tid; idx < nparts * kM * 4; idx += kTcThreads) {
      const int part = idx / (kM * 4), rem = idx % (kM * 4);
      const int m = rem / 4, c = rem % 4;
      const int x = (part < 2 ? ca : cb) + m;
      const int k = k0 + 8 * c;
      const bool ok = x >= 0 && x < J && k < w;
      const void* src = ok ? (const void*)(X2s + 2 * (int64_t)x * wp + ((part & 1) ? wp : 0) + k) : safe;
      const uint32_t dst = s0 + part * Cfg<2>::kOp + (m >> 3) * 512 + (m & 7) * 64 + ((c ^ ((m >> 1) & 3)) << 4);
      cp_async16(dst, src, ok);
    }
  }
}

template <int SPLIT>
__global__ void __launch_bounds__(kTcThreads, SPLIT == 2 ? 2 : 1) syrk_tc_kernel(DevPlan P, const int2* items, int nitems,
                                                                const float* X, const uint16_t* X2, float* F,
                                                                int* status) {
  using C = Cfg<SPLIT>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t mbar[kStages];
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  __shared__ Meta meta[kMetaCap];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = idesc_mn128(SPLIT ? 1u : 2u);
  constexpr int kOpB = Cfg<SPLIT>::kOp;
  uint32_t g0 = 0;  // chunks issued by this CTA so far (stage = g % kStages)

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int si = items[it].x, t2 = items[it].y;
    const SubInfo S = P.sub[si];
    int BI, BJ;
    tile2_of(t2, BI, BJ);
    const int* tl = P.t2_off + S.t20;
    const int cbeg = tl[t2], cend = tl[t2 + 1];
    // the tile's contributing blocks, staged once (the chunk loop then reads no dependent global data)
    auto meta_of = [&](int c) {
      const int s = P.t2_sn[c];
      const int gs = S.sn0 + s, bs = S.bsn0 + s;
      Meta m;
      m.w = P.sn_w[gs];
      m.wp = (m.w + 7) & ~7;
      m.jb = P.jb[bs];
      m.J = P.je[bs] - m.jb;
      m.xofs = P.Xofs[bs];
      return m;
    };
    const bool staged = cend - cbeg <= kMetaCap;
    if (staged)
      for (int c = cbeg + tid; c < cend; c += kTcThreads) meta[c - cbeg] = meta_of(c);
    __syncthreads();
    int nch = 0;
    for (int c = cbeg; c < cend; ++c) {
      const int w = staged ? meta[c - cbeg].w : P.sn_w[S.sn0 + P.t2_sn[c]];
      nch += (w + C::kKC - 1) / C::kKC;
    }
    const float* Xsub = X + S.X;
    const uint16_t* X2sub = X2 + 2 * S.X;
    const bool diag = BI == BJ;
    Cursor cur{cbeg, 0};
    auto issue = [&](int i) {
      // load local chunk i (the cursor walks the chunks in order)
      const Meta m = staged ? meta[cur.c - cbeg] : meta_of(cur.c);
      uint8_t* stage = smem + ((g0 + i) % kStages) * C::kStageBytes;
      load_chunk<SPLIT>(stage, Xsub + m.xofs, X2sub + 2 * m.xofs, m.wp, m.w, m.J, BI * kM - m.jb, BJ * kM - m.jb,
                        cur.k0, SPLIT ? (const void*)X2 : (const void*)X, diag);
      cur.k0 += C::kKC;
      if (cur.k0 >= m.w) {
        cur.c++;
        cur.k0 = 0;
      }
    };
    for (int i = 0; i < nch + kStages - 1; ++i) {
      if (i < nch) {
        if (i >= kStages) {
          const uint32_t gp = g0 + i - kStages;
          if (tid == 0 && !mbar_wait(smem_u32(&mbar[gp % kStages]), (gp / kStages) & 1)) s_abort = 1;
          __syncthreads();
          if (s_abort) break;
        }
        issue(i);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      const int j = i - (kStages - 1);
      if (j >= 0 && j < nch) {
        asm volatile("cp.async.wait_group %0;" ::"n"(kStages - 1) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sbase = smem_u32(smem + ((g0 + j) % kStages) * C::kStageBytes);
          if constexpr (!SPLIT) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ad = sw128_desc(sbase + kk * 32), bd = sw128_desc(sbase + kOpBytes + kk * 32);
              mma_tf32(tmem, ad, bd, idesc, (j > 0 || kk > 0) ? 1u : 0u);
            }
          } else {
#pragma unroll
            for (int kk = 0; kk < C::kKC / 16; ++kk) {
              const uint32_t o = kk * 32;
              auto dsc = [](uint32_t a) { return SPLIT == 2 ? sw64_desc(a) : sw128_desc(a); };
              const uint64_t ah = dsc(sbase + o), al = dsc(sbase + kOpB + o);
              const uint64_t bh = diag ? ah : dsc(sbase + 2 * kOpB + o);
              const uint64_t bl = diag ? al : dsc(sbase + 3 * kOpB + o);
              mma_f16(tmem, ah, bh, idesc, (j > 0 || kk > 0) ? 1u : 0u);
              mma_f16(tmem, ah, bl, idesc, 1u);
              mma_f16(tmem, al, bh, idesc, 1u);
            }
          }
          mma_commit(smem_u32(&mbar[(g0 + j) % kStages]));
        }
      }
    }
    if (s_abort) break;
    if (nch > 0) {
      const uint32_t gl = g0 + nch - 1;
      if (tid == 0 && !mbar_wait(smem_u32(&mbar[gl % kStages]), (gl / kStages) & 1)) s_abort = 1;
      __syncthreads();
      if (s_abort) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    g0 += nch;
    // epilogue: warp w owns tile rows 32 (w % 4) .. + 31 (its TMEM lane quarter) and the column chunks
    // 2 (w / 4), 2 (w / 4) + 1 of 32 columns
    const int quarter = warp % 4;
    const int row = BI * kM + quarter * 32 + lane;
    const int bi = row / kT;
#pragma unroll 1
    for (int cc = 2 * (warp / 4); cc < 2 * (warp / 4) + 2; ++cc) {
      uint32_t v[32];
      if (nch > 0) {
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + cc * 32, v);
      } else {
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = 0u;
      }
      const int col = BJ * kM + cc * 32;
      const int bj = col / kT;
      if (bi < S.nb && bj < S.nb && bj <= bi && (row % kT) < tile_rows(S.nb, S.vr, bi)) {
        float* tb = F + S.F + tile_offset<4>(S.nb, S.vr, bi, bj);
        const int r = row % kT;
        if (bj < bi) {
#pragma unroll
          for (int e = 0; e < 32; e += 4)
            *reinterpret_cast<float4*>(tb + tile_pos(r, col % kT + e)) =
                make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]), __uint_as_float(v[e + 2]),
                            __uint_as_float(v[e + 3]));
        } else {
          // diagonal tile: the chunks up to the one holding column r, zeros right of the diagonal
#pragma unroll
          for (int e = 0; e < 32; e += 4) {
            const int c = col % kT + e;
            if (c / 4 <= r / 4) {
              float x[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) x[u] = c + u <= r ? __uint_as_float(v[e + u]) : 0.f;
              *reinterpret_cast<float4*>(tb + diag_pos<4>(r, c)) = make_float4(x[0], x[1], x[2], x[3]);
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  // drain copies, release TMEM
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (s_abort && tid == 0) atomicOr(status, kStatTimeout);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

// ---------------------------------------------------------------- warp-specialised split-bf16 SYRK
//
// The same tiles, K chunks and operand layout as syrk_tc_kernel<1>, with the roles split so that loads, MMAs
// and the write-back overlap: four producer warps keep kWsStages chunks of cp.async copies in flight (each
// thread waits for its own oldest group, fences it for the tensor cores and arrives on that stage's "full"
// barrier), one thread issues the MMAs of a chunk once its stage is full and commits them to the stage's
// "empty" barrier, and four epilogue warps drain a double-buffered TMEM accumulator (tile t uses columns
// 128 (t mod 2) ..) while the next tile is multiplied.  Every wait is bounded; a timeout stops all roles,
// the issuer waits for its MMAs, TMEM is freed and kStatTimeout is reported.
constexpr int kWsProd = 4;                                 // producer warps
constexpr int kWsThreads = 32 * (kWsProd + 1 + 4);         // producers, MMA issuer, epilogue
constexpr int kWsStages = 3;
constexpr uint32_t kWsTmemCols = 256;                      // two 128-column accumulators
constexpr int kWsStageBytes = 4 * kOpBytes;                // A hi, A lo, B hi, B lo

// wait on an mbarrier phase, giving up on a timeout (flagged) or when another role has given up
__device__ __forceinline__ bool ws_wait(uint32_t mbar, uint32_t parity, volatile int* abort) {
  for (int i = 0; i < (1 << 25); ++i) {
    if (mbar_test(mbar, parity)) return true;
    if (*abort) return false;
    __nanosleep(32);
  }
  *abort = 1;
  return false;
}

__global__ void __launch_bounds__(kWsThreads, 1) syrk_ws_kernel(DevPlan P, const int2* items, int nitems,
                                                               const uint16_t* X2, float* F, int* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[kWsStages], empty[kWsStages], accf[2], acce[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;
  __shared__ int p_stop;  // the producers' copy of s_abort, read by all of them between two barriers
  __shared__ Meta meta[kMetaCap];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  constexpr int kProdThreads = 32 * kWsProd;

  if (warp == kWsProd) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kWsTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int k = 0; k < kWsStages; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[k])), "r"(kProdThreads));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[k])));
    }
    for (int a = 0; a < 2; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf[a])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acce[a])), "r"(128));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&drain)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp < kWsProd) {
    // ------------------------------------------------ producers
    uint32_t cg = 0;  // chunks issued by this CTA
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
      // every producer thread passes the named barrier equally often: the stop decision is taken between
      // two barriers from one read of the flag
      asm volatile("bar.sync 1, %0;" ::"n"(kProdThreads) : "memory");
      if (tid == 0) p_stop = s_abort;
      asm volatile("bar.sync 1, %0;" ::"n"(kProdThreads) : "memory");
      if (p_stop) break;
      const int si = items[it].x, t2 = items[it].y;
      const SubInfo S = P.sub[si];
      int BI, BJ;
      tile2_of(t2, BI, BJ);
      const int* tl = P.t2_off + S.t20;
      const int cbeg = tl[t2], cend = tl[t2 + 1];
      auto meta_of = [&](int c) {
        const int sn = P.t2_sn[c];
        const int gs = S.sn0 + sn, bs = S.bsn0 + sn;
        Meta m;
        m.w = P.sn_w[gs];
        m.wp = (m.w + 7) & ~7;
        m.jb = P.jb[bs];
        m.J = P.je[bs] - m.jb;
        m.xofs = P.Xofs[bs];
        return m;
      };
      const bool staged = cend - cbeg <= kMetaCap;
      // (the barriers above also order the previous tile's reads of meta before these writes)
      if (staged)
        for (int c = cbeg + tid; c < cend; c += kProdThreads) meta[c - cbeg] = meta_of(c);
      asm volatile("bar.sync 1, %0;" ::"n"(kProdThreads) : "memory");
      const uint16_t* X2sub = X2 + 2 * S.X;
      const bool diag = BI == BJ;
      const int nparts = diag ? 2 : 4;
      for (int c = cbeg; c < cend && !s_abort; ++c) {
        const Meta m = staged ? meta[c - cbeg] : meta_of(c);
        const uint16_t* X2s = X2sub + 2 * m.xofs;
        const int ca = BI * kM - m.jb, cbb = BJ * kM - m.jb;
        for (int k0 = 0; k0 < m.w; k0 += 64, ++cg) {
          const int st = (int)(cg % kWsStages);
          if (cg >= kWsStages && !ws_wait(smem_u32(&empty[st]), ((cg / kWsStages) - 1) & 1, &s_abort)) break;
          const uint32_t s0 = smem_u32(smem + st * kWsStageBytes);
          for (int idx = tid; idx < nparts * kM * 8; idx += kProdThreads) {
            const int part = idx / (kM * 8), rem = idx % (kM * 8);
            const int mrow = rem / 8, c8 = rem % 8;
            const int x = (part < 2 ? ca : cbb) + mrow;
            const int k = k0 + 8 * c8;
            const bool ok = x >= 0 && x < m.J && k < m.w;
            const void* src = ok ? (const void*)(X2s + 2 * (int64_t)x * m.wp + ((part & 1) ? m.wp : 0) + k)
                                 : (const void*)X2;
            cp_async16(s0 + part * kOpBytes + (mrow >> 3) * 1024 + (mrow & 7) * 128 + ((c8 ^ (mrow & 7)) << 4), src,
                       ok);
          }
          asm volatile("cp.async.commit_group;" ::: "memory");
          if (cg >= kWsStages - 1) {
            // this thread's copies of chunk cg - (kWsStages - 1) have landed: fence them for the tensor cores
            asm volatile("cp.async.wait_group %0;" ::"n"(kWsStages - 1) : "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[(cg - (kWsStages - 1)) %
                                                                                            kWsStages])));
          }
        }
      }
    }
    // the last chunks
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const uint32_t nout = cg < (uint32_t)(kWsStages - 1) ? cg : (uint32_t)(kWsStages - 1);
    for (uint32_t k = cg - nout; k < cg; ++k)
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[k % kWsStages])));
  } else if (warp == kWsProd) {
    // ------------------------------------------------ MMA issuer (lane 0; the warp computes the chunk counts)
    constexpr uint32_t idesc = idesc_mn128(1u);
    uint32_t cg = 0, tl_count = 0;
    bool issued = false;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x, ++tl_count) {
      if (__shfl_sync(0xffffffffu, (int)s_abort, 0)) break;  // one decision for the whole warp
      const int si = items[it].x, t2 = items[it].y;
      const SubInfo S = P.sub[si];
      int BI, BJ;
      tile2_of(t2, BI, BJ);
      const int* tl = P.t2_off + S.t20;
      const int cbeg = tl[t2], cend = tl[t2 + 1];
      int nch = 0;
      for (int c = cbeg + lane; c < cend; c += 32) nch += (P.sn_w[S.sn0 + P.t2_sn[c]] + 63) / 64;
      for (int o = 16; o > 0; o >>= 1) nch += __shfl_xor_sync(0xffffffffu, nch, o);
      const bool diag = BI == BJ;
      const uint32_t a = tl_count % 2;
      if (lane == 0) {
        bool ok = true;
        if (tl_count >= 2) ok = ws_wait(smem_u32(&acce[a]), ((tl_count / 2) - 1) & 1, &s_abort);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + a * 128;
        for (int i = 0; i < nch && ok; ++i, ++cg) {
          const int st = (int)(cg % kWsStages);
          if (!ws_wait(smem_u32(&full[st]), (cg / kWsStages) & 1, &s_abort)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sbase = smem_u32(smem + st * kWsStageBytes);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t o = kk * 32;
            const uint64_t ah = sw128_desc(sbase + o), al = sw128_desc(sbase + kOpBytes + o);
            const uint64_t bh = diag ? ah : sw128_desc(sbase + 2 * kOpBytes + o);
            const uint64_t bl = diag ? al : sw128_desc(sbase + 3 * kOpBytes + o);
            mma_f16(d, ah, bh, idesc, (i > 0 || kk > 0) ? 1u : 0u);
            mma_f16(d, ah, bl, idesc, 1u);
            mma_f16(d, al, bh, idesc, 1u);
          }
          mma_commit(smem_u32(&empty[st]));
          issued = true;
        }
        mma_commit(smem_u32(&accf[a]));  // the tile's accumulator is complete (at once if nothing was issued)
      }
      __syncwarp();
    }
    if (lane == 0 && issued) {
      // every MMA has completed before TMEM is released (also after a timeout)
      mma_commit(smem_u32(&drain));
      if (!mbar_wait(smem_u32(&drain), 0)) s_abort = 1;
    }
  } else {
    // ------------------------------------------------ epilogue: TMEM lane quarter warp % 4, all 128 columns
    const int quarter = warp % 4;
    uint32_t tl_count = 0;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x, ++tl_count) {
      const int si = items[it].x, t2 = items[it].y;
      const SubInfo S = P.sub[si];
      int BI, BJ;
      tile2_of(t2, BI, BJ);
      const int* tl = P.t2_off + S.t20;
      const bool empty_tile = tl[t2 + 1] == tl[t2];
      const uint32_t a = tl_count % 2;
      // lane 0 waits, the warp follows its outcome (tcgen05.ld below needs every lane)
      int ok = 0;
      if (lane == 0) ok = ws_wait(smem_u32(&accf[a]), (tl_count / 2) & 1, &s_abort) ? 1 : 0;
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = BI * kM + quarter * 32 + lane;
      const int bi = row / kT;
#pragma unroll 1
      for (int cc = 0; cc < 4; ++cc) {
        uint32_t v[32];
        if (!empty_tile) {
          tmem_ld32(tmem + a * 128 + ((uint32_t)(quarter * 32) << 16) + cc * 32, v);
        } else {
#pragma unroll
          for (int e = 0; e < 32; ++e) v[e] = 0u;
        }
        const int col = BJ * kM + cc * 32;
        const int bj = col / kT;
        if (bi < S.nb && bj < S.nb && bj <= bi && (row % kT) < tile_rows(S.nb, S.vr, bi)) {
          float* tb = F + S.F + tile_offset<4>(S.nb, S.vr, bi, bj);
          const int r = row % kT;
          if (bj < bi) {
#pragma unroll
            for (int e = 0; e < 32; e += 4)
              *reinterpret_cast<float4*>(tb + tile_pos(r, col % kT + e)) =
                  make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]), __uint_as_float(v[e + 2]),
                              __uint_as_float(v[e + 3]));
          } else {
#pragma unroll
            for (int e = 0; e < 32; e += 4) {
              const int c = col % kT + e;
              if (c / 4 <= r / 4) {
                float x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = c + u <= r ? __uint_as_float(v[e + u]) : 0.f;
                *reinterpret_cast<float4*>(tb + diag_pos<4>(r, c)) = make_float4(x[0], x[1], x[2], x[3]);
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[a])));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (s_abort && tid == 0) atomicOr(status, kStatTimeout);
  if (warp == kWsProd) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWsTmemCols));
  }
}

}  // namespace

size_t syrk_tc_smem(int split) {
  return (size_t)kStages * (split == 2 ? Cfg<2>::kStageBytes : split ? Cfg<1>::kStageBytes : Cfg<0>::kStageBytes) +
         1024;
}

void launch_syrk_tc(const DevPlan& P, const int2* items, int nitems, const float* X, const uint16_t* X2, float* F,
                    int grid, int split, int* status, cudaStream_t st, int variant) {
  size_t smem = syrk_tc_smem(split && variant == 2 ? 2 : split);
  if (split && variant == 2) {
    cudaFuncSetAttribute(syrk_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    syrk_tc_kernel<2><<<grid, kTcThreads, smem, st>>>(P, items, nitems, X, X2, F, status);
  } else if (split && variant == 1) {
    const int ws_smem = kWsStages * kWsStageBytes + 1024;
    cudaFuncSetAttribute(syrk_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ws_smem);
    syrk_ws_kernel<<<grid, kWsThreads, ws_smem, st>>>(P, items, nitems, X2, F, status);
  } else if (split) {
    cudaFuncSetAttribute(syrk_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    syrk_tc_kernel<1><<<grid, kTcThreads, smem, st>>>(P, items, nitems, X, X2, F, status);
  } else {
    cudaFuncSetAttribute(syrk_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    syrk_tc_kernel<0><<<grid, kTcThreads, smem, st>>>(P, items, nitems, X, X2, F, status);
  }
}

}  // namespace feti
