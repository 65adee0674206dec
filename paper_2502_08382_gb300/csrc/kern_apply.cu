// Explicit application q = F p (paper eq. 12 summed over subdomains, with
// Algorithm 2's scatter / per-subdomain apply / gather), three launches:
//
//  0. scatter: pg[j] = p[map_i(j)] for every sorted column j of every
//             subdomain (Algorithm 2's scatter), in the tile precision;
//  1. tiles:  every warp streams whole F tiles from HBM straight into
//             registers with 16-byte coalesced loads (each warp-wide load
//             covers 512 contiguous bytes: two FP32 rows or one FP64 row),
//             keeping two batches of BATCH loads in flight (only the batches
//             that hold stored rows), and writes per tile t the row partial
//             F_t p_bj (row slot t, stored rows only) and the column
//             partial F_t^T p_bi (column slot t; for a diagonal tile only its
//             strictly lower part, transposed).  Tiles are dealt to warps
//             round-robin, so all warps stream neighbouring tiles together
//             and the load is balanced to one tile;
//  2. gather: q[lambda] = sum over the (at most two) subdomain columns of
//             lambda of that column's tile partials (the row partials of its
//             tile row and the column partials of its tile column), in FP64
//             and in a fixed order (deterministic, no atomics).
// Tile arithmetic runs in the tile's precision (FP32 tiles: FP32 FMAs); the
// cross-tile sums in phase 2 are FP64.  Nothing waits on another warp.
#include <algorithm>
#include <mutex>

#include "feti.h"
#include "common.cuh"
#include "kernels.h"

namespace feti {
namespace {

constexpr int kApplyThreads = 128;

template <typename TF>
struct Vec16;
template <>
struct Vec16<float> {
  using T = float4;
};
template <>
struct Vec16<double> {
  using T = double2;
};

__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ double2 ld_stream(const double2* p) { return __ldcs(p); }

// Per loaded 16-byte chunk v of a tile row: the row-dot part v . pc, and the
// column partials cacc += v * pr.  FP32 uses the packed two-wide FMA of
// sm_100+ (half the instructions of the scalar form; the column partials
// round exactly as scalar FMAs would).
__device__ __forceinline__ float dot16(const float4& v, const float4& pc) {
  float2 d = __fmul2_rn(make_float2(v.x, v.y), make_float2(pc.x, pc.y));
  d = __ffma2_rn(make_float2(v.z, v.w), make_float2(pc.z, pc.w), d);
  return d.x + d.y;
}
__device__ __forceinline__ double dot16(const double2& v, const double2& pc) { return fma(v.y, pc.y, v.x * pc.x); }
__device__ __forceinline__ void axpy16(const float4& v, float pr, float* cacc) {
  const float2 pp = make_float2(pr, pr);
  const float2 c01 = __ffma2_rn(make_float2(v.x, v.y), pp, make_float2(cacc[0], cacc[1]));
  const float2 c23 = __ffma2_rn(make_float2(v.z, v.w), pp, make_float2(cacc[2], cacc[3]));
  cacc[0] = c01.x;
  cacc[1] = c01.y;
  cacc[2] = c23.x;
  cacc[3] = c23.y;
}
__device__ __forceinline__ void axpy16(const double2& v, double pr, double* cacc) {
  cacc[0] = fma(v.x, pr, cacc[0]);
  cacc[1] = fma(v.y, pr, cacc[1]);
}
// v with the components at column >= r (right of the diagonal of row r) set to zero
__device__ __forceinline__ float4 mask_diag(const float4& v, int c0, int r) {
  return make_float4(c0 < r ? v.x : 0.f, c0 + 1 < r ? v.y : 0.f, c0 + 2 < r ? v.z : 0.f, c0 + 3 < r ? v.w : 0.f);
}
__device__ __forceinline__ double2 mask_diag(const double2& v, int c0, int r) {
  return make_double2(c0 < r ? v.x : 0.0, c0 + 1 < r ? v.y : 0.0);
}

template <typename TF>
__global__ void scatter_kernel(const int* qmap, int64_t ncols, const double* p, TF* pg) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ncols; g += (int64_t)gridDim.x * blockDim.x) {
    const int lam = qmap[g];
    pg[g] = lam >= 0 ? (TF)p[lam] : (TF)0;
  }
}

// Reduce-scatter of N values per lane over the lanes that differ in bits
// O, O/2, ..., 1 of the lane index: while N > 1 each step keeps half of the
// values (the upper half where the lane's bit is set) and adds the partner's
// other half; once one value is left, the remaining steps add it outright.
// Afterwards lane l holds, in v[0], the total of value index
// (l mod 2O) >> log2(2O / N_initial) (for N_initial <= 2O).
template <typename TF, int N, int O>
struct ReduceScatter {
  __device__ __forceinline__ static void run(TF* v, int lane) {
    if constexpr (O >= 1) {
      if constexpr (N > 1) {
        const bool up = (lane & O) != 0;
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
          const TF send = up ? v[i] : v[i + N / 2];
          const TF keep = up ? v[i + N / 2] : v[i];
          v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
        }
        ReduceScatter<TF, N / 2, O / 2>::run(v, lane);
      } else {
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], O);
        ReduceScatter<TF, 1, O / 2>::run(v, lane);
      }
    }
  }
};

// Per-buffer state of one issued batch.
template <typename TF, int BATCH>
struct Batch {
  typename Vec16<TF>::T v[BATCH];
  typename Vec16<TF>::T pc;  // p of the tile's column block, this lane's chunk
  TF pr;                     // p of one row of the batch (shuffled out per load)
  int t, b, rows, diag;
};

template <typename TF, int BATCH>
struct TileStream {
  using VT = typename Vec16<TF>::T;
  static constexpr int V = 16 / (int)sizeof(TF);  // values per 16-byte chunk
  static constexpr int NCH = kT / V;              // lanes per tile row
  static constexpr int RPL = 32 / NCH;            // rows per warp-wide load
  static constexpr int ROWS_B = BATCH * RPL;      // rows per batch
  static constexpr int NBT = kT / ROWS_B;         // batches per tile
  static_assert(NBT >= 1 && kT % ROWS_B == 0, "batch does not divide a tile");

  const TileDesc* desc;
  const TF* F;
  const TF* pg;
  int lane, cq, half, gw, nw, ntiles;
  TileDesc dI;    // descriptor of the tile being issued
  TileDesc dP;    // prefetched descriptor of the next tile of this warp

  // Item k of this warp = batch k % NBT of its tile k / NBT.  A batch that lies
  // entirely below the stored rows (the ragged last block row) issues no load.
  __device__ __forceinline__ void issue(int k, Batch<TF, BATCH>& B) {
    const int j = k / NBT, b = k % NBT;
    const int t = gw + j * nw;
    if (b == 0 && k > 0) {
      dI = dP;
      const int tn = t + nw;
      if (tn < ntiles) dP = desc[tn];
    }
    const TileDesc& d = dI;
    const bool diag = (d.flags & kTileDiag) != 0;
    B.t = d.slot;
    B.b = b;
    B.rows = d.rows;
    B.diag = diag;
    if (b * ROWS_B >= d.rows) return;  // empty batch (warp-uniform)
    const TF* Ft = F + d.f_ofs;
    if (!diag && d.rows == kT) {
#pragma unroll
      for (int i = 0; i < BATCH; ++i) {
        const int r = b * ROWS_B + i * RPL + half;
        B.v[i] = ld_stream(reinterpret_cast<const VT*>(Ft + r * kT + cq * V));
      }
    } else {
      // ragged or diagonal tile: only stored positions are loaded
#pragma unroll
      for (int i = 0; i < BATCH; ++i) {
        const int r = b * ROWS_B + i * RPL + half;
        const bool ok = r < d.rows && (!diag || cq * V <= r);
        const int64_t off = diag ? diag_row_off<(int)sizeof(TF)>(r) : (int64_t)r * kT;
        if (ok) B.v[i] = ld_stream(reinterpret_cast<const VT*>(Ft + off + cq * V));
        else B.v[i] = VT{};
      }
    }
    B.pc = *reinterpret_cast<const VT*>(pg + d.pcol + cq * V);
    B.pr = pg[d.prow + b * ROWS_B + (lane % ROWS_B)];
  }
};

template <typename TF, int BATCH>
__device__ __forceinline__ void consume(const Batch<TF, BATCH>& B, TF* cacc, TF* rowpart, TF* colpart, int lane,
                                        int cq, int half) {
  using TS = TileStream<TF, BATCH>;
  constexpr int V = TS::V, NCH = TS::NCH, RPL = TS::RPL, ROWS_B = TS::ROWS_B, NBT = TS::NBT;
  if (B.b * ROWS_B < B.rows) {
    TF rs[BATCH];
    if (B.diag) {
      // the stored chunk of a diagonal row holds zeros right of the diagonal; the column
      // partials must also leave out the diagonal itself (it is the row partial's)
#pragma unroll
      for (int i = 0; i < BATCH; ++i) {
        const TF pr = __shfl_sync(0xffffffffu, B.pr, i * RPL + half);
        const int r = B.b * ROWS_B + i * RPL + half;
        rs[i] = dot16(B.v[i], B.pc);
        axpy16(mask_diag(B.v[i], cq * V, r), pr, cacc);
      }
    } else {
#pragma unroll
      for (int i = 0; i < BATCH; ++i) {
        const TF pr = __shfl_sync(0xffffffffu, B.pr, i * RPL + half);
        rs[i] = dot16(B.v[i], B.pc);
        axpy16(B.v[i], pr, cacc);
      }
    }
    ReduceScatter<TF, BATCH, NCH / 2>::run(rs, lane);
    constexpr int SPAN = NCH / BATCH;  // lanes holding the same row total
    if (cq % SPAN == 0) {
      const int r = B.b * ROWS_B + (cq / SPAN) * RPL + half;
      // rows beyond the stored ones are padding columns of q_i, never gathered: not written
      if (r < B.rows) rowpart[(int64_t)B.t * kT + r] = rs[0];
    }
  }
  if (B.b == NBT - 1) {
    if constexpr (RPL == 2) {
#pragma unroll
      for (int e = 0; e < V; ++e) cacc[e] += __shfl_xor_sync(0xffffffffu, cacc[e], 16);
    }
    if (half == 0) {
      using VT = typename Vec16<TF>::T;
      VT o;
      if constexpr (V == 4) o = VT{cacc[0], cacc[1], cacc[2], cacc[3]};
      else o = VT{cacc[0], cacc[1]};
      *reinterpret_cast<VT*>(colpart + (int64_t)B.t * kT + cq * V) = o;
    }
#pragma unroll
    for (int e = 0; e < V; ++e) cacc[e] = (TF)0;
  }
}

template <typename TF, int BATCH>
__global__ void __launch_bounds__(kApplyThreads) apply_tiles_kernel(const TileDesc* __restrict__ desc, int ntiles,
                                                                   const TF* __restrict__ F,
                                                                   const TF* __restrict__ pg, TF* rowpart,
                                                                   TF* colpart, const int* active) {
  if (active && *active == 0) return;  // the iteration this launch belongs to has stopped
  using TS = TileStream<TF, BATCH>;
  constexpr int V = TS::V, NBT = TS::NBT;
  TS ts;
  ts.desc = desc;
  ts.F = F;
  ts.pg = pg;
  ts.lane = threadIdx.x & 31;
  ts.cq = ts.lane % TS::NCH;
  ts.half = ts.lane / TS::NCH;
  ts.nw = gridDim.x * (blockDim.x / 32);
  ts.gw = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  ts.ntiles = ntiles;
  if (ts.gw >= ntiles) return;
  const int my_tiles = (ntiles - 1 - ts.gw) / ts.nw + 1;
  const int nitems = my_tiles * NBT;
  ts.dI = desc[ts.gw];
  ts.dP = ts.gw + ts.nw < ntiles ? desc[ts.gw + ts.nw] : ts.dI;
  TF cacc[V];
#pragma unroll
  for (int e = 0; e < V; ++e) cacc[e] = (TF)0;
  Batch<TF, BATCH> b0, b1;
  ts.issue(0, b0);
  int k = 0;
  for (;;) {
    if (k + 1 < nitems) ts.issue(k + 1, b1);
    consume<TF, BATCH>(b0, cacc, rowpart, colpart, ts.lane, ts.cq, ts.half);
    if (++k >= nitems) break;
    if (k + 1 < nitems) ts.issue(k + 1, b0);
    consume<TF, BATCH>(b1, cacc, rowpart, colpart, ts.lane, ts.cq, ts.half);
    if (++k >= nitems) break;
  }
}

// ---------------------------------------------------------------- bulk-copy ring variant
//
// Every warp runs its own ring of S shared-memory stages.  A stage holds one
// batch of one tile: the batch's stored rows (contiguous in F: one bulk copy),
// the tile's column-block p and the batch's row p values.  Lane 0 arms the
// stage's mbarrier with the byte count and issues the three copies; the warp
// waits on the barrier (bounded), computes from shared memory, and re-arms the
// stage with the item S ahead.  The copy engine does the address work and the
// data in flight needs no registers.  No warp waits on another.

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// every lane polls the barrier phase (bounded, about a second), so that each one
// observes the completed copies; true only if the whole warp saw the phase complete
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  int ok = 0;
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) {
      ok = 1;
      break;
    }
    if (clock64() - t0 > 2000000000LL) break;
  }
  return __all_sync(0xffffffffu, ok) != 0;
}

template <typename TF>
struct RingCfg {
  static constexpr int V = 16 / (int)sizeof(TF);
  static constexpr int NCH = kT / V;
  static constexpr int RPL = 32 / NCH;
  static constexpr int BATCH = 16;
  static constexpr int ROWS_B = BATCH * RPL;            // 32 (FP32) / 16 (FP64) rows per stage
  static constexpr int DATA = ROWS_B * kT * (int)sizeof(TF);  // 8 KB
  static constexpr int PC = kT * (int)sizeof(TF);
  static constexpr int PR = ROWS_B * (int)sizeof(TF);
  static constexpr int STAGE = DATA + PC + PR;          // multiple of 16 bytes
  __host__ __device__ static constexpr size_t bars_ofs(int W, int S) { return (size_t)W * S * STAGE; }
  __host__ __device__ static constexpr size_t meta_ofs(int W, int S) { return (bars_ofs(W, S) + (size_t)W * S * 8 + 15) / 16 * 16; }
  __host__ __device__ static constexpr size_t smem(int W, int S) { return meta_ofs(W, S) + (size_t)W * S * 16 + 128; }
};

// Position of a warp in its sequence of (tile, batch) items: tiles gw, gw + nw,
// ..., and inside a tile only the batches that hold stored rows.
struct RingCursor {
  int t, b;
  TileDesc d;   // descriptor of tile t
  TileDesc dn;  // prefetched descriptor of tile t + nw
};

template <int ROWS_B>
__device__ __forceinline__ bool ring_advance(RingCursor& c, int nw, int ntiles, const TileDesc* desc) {
  if ((c.b + 1) * ROWS_B < c.d.rows) {
    ++c.b;
    return true;
  }
  c.t += nw;
  c.b = 0;
  if (c.t >= ntiles) return false;
  c.d = c.dn;
  if (c.t + nw < ntiles) c.dn = desc[c.t + nw];
  return true;
}

template <typename TF, int W, int S>
__global__ void __launch_bounds__(W * 32) apply_ring_kernel(const TileDesc* __restrict__ desc, int ntiles,
                                                            const TF* __restrict__ F, const TF* __restrict__ pg,
                                                            TF* rowpart, TF* colpart, const int* active,
                                                            int* status) {
  if (active && *active == 0) return;
  using C = RingCfg<TF>;
  using VT = typename Vec16<TF>::T;
  constexpr int V = C::V, NCH = C::NCH, RPL = C::RPL, BATCH = C::BATCH, ROWS_B = C::ROWS_B;
  extern __shared__ __align__(128) uint8_t ring_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cq = lane % NCH, half = lane / NCH;
  const int nw = gridDim.x * W, gw = blockIdx.x * W + warp;
  if (gw >= ntiles) return;  // whole warp; warps own their rings, nothing is shared
  uint8_t* ring = ring_smem + (size_t)warp * S * C::STAGE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(ring_smem + C::bars_ofs(W, S)) + warp * S;
  int4* meta = reinterpret_cast<int4*>(ring_smem + C::meta_ofs(W, S)) + warp * S;
  if (lane == 0) {
    for (int k = 0; k < S; ++k) bar_init(&bars[k]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  RingCursor ic;
  ic.t = gw;
  ic.b = 0;
  ic.d = desc[gw];
  ic.dn = gw + nw < ntiles ? desc[gw + nw] : ic.d;
  bool more = true;
  int issued = 0, consumed = 0;
  auto issue = [&](int slot) {
    if (lane == 0) {
      const TileDesc& d = ic.d;
      const bool diag = (d.flags & kTileDiag) != 0;
      const int r0 = ic.b * ROWS_B, r1 = min(r0 + ROWS_B, d.rows);
      const int64_t e0 = diag ? diag_row_off<(int)sizeof(TF)>(r0) : (int64_t)r0 * kT;
      const int64_t e1 = diag ? diag_row_off<(int)sizeof(TF)>(r1) : (int64_t)r1 * kT;
      const uint32_t bytes = (uint32_t)((e1 - e0) * (int64_t)sizeof(TF));
      uint8_t* st = ring + (size_t)slot * C::STAGE;
      meta[slot] = make_int4(d.slot, ic.b, d.rows, diag ? 1 : 0);
      bar_expect(&bars[slot], bytes + C::PC + C::PR);
      bulk_to_smem(st, F + d.f_ofs + e0, bytes, &bars[slot]);
      bulk_to_smem(st + C::DATA, pg + d.pcol, C::PC, &bars[slot]);
      bulk_to_smem(st + C::DATA + C::PC, pg + d.prow + r0, C::PR, &bars[slot]);
    }
  };
  for (; issued < S && more; ++issued) {
    issue(issued);
    more = ring_advance<ROWS_B>(ic, nw, ntiles, desc);
  }
  __syncwarp();  // lane 0's stage metadata is visible to the warp
  TF cacc[V];
#pragma unroll
  for (int e = 0; e < V; ++e) cacc[e] = (TF)0;
  bool failed = false;
  while (consumed < issued) {
    const int slot = consumed % S;
    if (!bar_wait(&bars[slot], (uint32_t)((consumed / S) & 1))) {
      failed = true;
      break;
    }
    const int4 mt = meta[slot];
    const int t = mt.x, b = mt.y, rows = mt.z;
    const bool diag = mt.w != 0;
    const uint8_t* st = ring + (size_t)slot * C::STAGE;
    const TF* sf = reinterpret_cast<const TF*>(st);
    const VT pc = *reinterpret_cast<const VT*>(st + C::DATA + cq * 16);
    const TF* prs = reinterpret_cast<const TF*>(st + C::DATA + C::PC);
    const int r0 = b * ROWS_B;
    const int64_t e0 = diag ? diag_row_off<(int)sizeof(TF)>(r0) : 0;
    TF rs[BATCH];
#pragma unroll
    for (int i = 0; i < BATCH; ++i) {
      const int r = r0 + i * RPL + half;
      const bool ok = r < rows && (!diag || cq * V <= r);
      const int64_t off = diag ? diag_row_off<(int)sizeof(TF)>(r) - e0 : (int64_t)(r - r0) * kT;
      const VT v = ok ? *reinterpret_cast<const VT*>(sf + off + cq * V) : VT{};
      const TF pr = prs[i * RPL + half];
      rs[i] = dot16(v, pc);
      axpy16(diag ? mask_diag(v, cq * V, r) : v, pr, cacc);
    }
    __syncwarp();  // the stage has been read by every lane: it may be refilled
    ++consumed;
    if (more) {
      issue(slot);
      ++issued;
      more = ring_advance<ROWS_B>(ic, nw, ntiles, desc);
    }
    ReduceScatter<TF, BATCH, NCH / 2>::run(rs, lane);
    constexpr int SPAN = NCH / BATCH;
    if (cq % SPAN == 0) {
      const int r = r0 + (cq / SPAN) * RPL + half;
      if (r < rows) rowpart[(int64_t)t * kT + r] = rs[0];
    }
    if (r0 + ROWS_B >= rows) {  // last batch of the tile
      if constexpr (RPL == 2) {
#pragma unroll
        for (int e = 0; e < V; ++e) cacc[e] += __shfl_xor_sync(0xffffffffu, cacc[e], 16);
      }
      if (half == 0) {
        VT o;
        if constexpr (V == 4) o = VT{cacc[0], cacc[1], cacc[2], cacc[3]};
        else o = VT{cacc[0], cacc[1]};
        *reinterpret_cast<VT*>(colpart + (int64_t)t * kT + cq * V) = o;
      }
#pragma unroll
      for (int e = 0; e < V; ++e) cacc[e] = (TF)0;
    }
  }
  if (failed) {
    // a copy did not land in time: report it and wait (bounded) for the copies still in flight
    if (lane == 0 && status) atomicOr(status, kStatTimeout);
    for (; consumed < issued; ++consumed) bar_wait(&bars[consumed % S], (uint32_t)((consumed / S) & 1));
  }
}

// q_i[b kT + x] = sum_{bj <= b} rowpart[tile (b, bj)][x] + sum_{bi >= b} colpart[tile (bi, b)][x];
// one warp per (subdomain, block), FP64 sums in a fixed order.
template <typename TF>
__global__ void reduce_tiles_kernel(DevPlan P, const int2* blocks, int nblocks, const TF* rowpart,
                                    const TF* colpart, double* qi, const int* active) {
  if (active && *active == 0) return;
  const int lane = threadIdx.x & 31;
  for (int wb = (blockIdx.x * blockDim.x + threadIdx.x) / 32; wb < nblocks; wb += gridDim.x * blockDim.x / 32) {
    const int2 sb = blocks[wb];
    const SubInfo& S = P.sub[sb.x];
    const int b = sb.y, nb = S.nb;
    const int64_t tb = S.tpart / kT;
    for (int x = lane; x < kT; x += 32) {
      double s = 0.0;
      const int64_t r0 = tb + (int64_t)b * (b + 1) / 2;
      for (int bj = 0; bj <= b; ++bj) s += (double)rowpart[(r0 + bj) * kT + x];
      for (int bi = b; bi < nb; ++bi) s += (double)colpart[(tb + (int64_t)bi * (bi + 1) / 2 + b) * kT + x];
      qi[S.qcol + (int64_t)b * kT + x] = s;
    }
  }
}

// q[lambda] = sum over its (at most two) subdomain columns of the tile partials
// of that column (tile_colsum), in subdomain order
template <typename TF>
__global__ void gather_tiles_kernel(DevPlan P, const int* colsub, const int* c0, const int* c1, int nlam,
                                    const TF* rowpart, const TF* colpart, double* q) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlam; l += gridDim.x * blockDim.x) {
    const int a = c0[l], b = c1[l];
    double s = a >= 0 ? tile_colsum(P.sub[colsub[a]], a, rowpart, colpart) : 0.0;
    if (b >= 0) s += tile_colsum(P.sub[colsub[b]], b, rowpart, colpart);
    q[l] = s;
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

template <typename TF, int BATCH>
void set_tiles_attr() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(apply_tiles_kernel<TF, BATCH>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    done = true;
  }
}

// variants of the tile kernel: register pipeline with 4 / 8 / 16-load batches
// (0, 1, 2), or per-warp bulk-copy rings of W warps x S stages: 4 x 3, 8 x 3, 2 x 6 (3, 4, 5)
constexpr int kRingW[3] = {4, 8, 2};
constexpr int kRingS[3] = {3, 3, 6};

template <typename TF, int W, int S>
void launch_ring(int grid, cudaStream_t st, const TileDesc* desc, int ntiles, const TF* F, const TF* pg, TF* rowpart,
                 TF* colpart, const int* active, int* status) {
  const size_t smem = RingCfg<TF>::smem(W, S);
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(apply_ring_kernel<TF, W, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    done = true;
  }
  apply_ring_kernel<TF, W, S><<<grid, W * 32, smem, st>>>(desc, ntiles, F, pg, rowpart, colpart, active, status);
}

template <typename TF>
void launch_tiles(int variant, int grid, cudaStream_t st, const TileDesc* desc, int ntiles, const TF* F,
                  const TF* pg, TF* rowpart, TF* colpart, const int* active = nullptr, int* status = nullptr) {
  if (ntiles <= 0) return;
  switch (variant) {
    case 0:
      set_tiles_attr<TF, 4>();
      apply_tiles_kernel<TF, 4><<<grid, kApplyThreads, 0, st>>>(desc, ntiles, F, pg, rowpart, colpart, active);
      break;
    case 1:
      set_tiles_attr<TF, 8>();
      apply_tiles_kernel<TF, 8><<<grid, kApplyThreads, 0, st>>>(desc, ntiles, F, pg, rowpart, colpart, active);
      break;
    case 2:
      set_tiles_attr<TF, 16>();
      apply_tiles_kernel<TF, 16><<<grid, kApplyThreads, 0, st>>>(desc, ntiles, F, pg, rowpart, colpart, active);
      break;
    case 3: launch_ring<TF, 4, 3>(grid, st, desc, ntiles, F, pg, rowpart, colpart, active, status); break;
    case 4: launch_ring<TF, 8, 3>(grid, st, desc, ntiles, F, pg, rowpart, colpart, active, status); break;
    default: launch_ring<TF, 2, 6>(grid, st, desc, ntiles, F, pg, rowpart, colpart, active, status); break;
  }
}

template <typename TF>
void launch_reduce(const DevPlan& P, const int2* blocks, int nblocks, const TF* rowpart, const TF* colpart,
                   double* qi, cudaStream_t st, const int* active = nullptr) {
  const int rg = std::max(1, std::min((nblocks + 7) / 8, 152 * 16));
  reduce_tiles_kernel<TF><<<rg, 256, 0, st>>>(P, blocks, nblocks, rowpart, colpart, qi, active);
}

}  // namespace

template <typename TF>
static void launch_apply_t(const DevPlan& P, const TileDesc* desc, int ntiles, const void* F, const int* qmap,
                           int64_t ncols, const double* p, void* pg, void* rowpart, void* colpart, const int2* blocks,
                           int nblocks, double* qi, const int* c0, const int* c1, int nlam, double* q, int grid,
                           int variant, int* status, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  const int sg = (int)std::max<int64_t>(1, std::min<int64_t>((ncols + 255) / 256, 152 * 8));
  scatter_kernel<TF><<<sg, 256, 0, st>>>(qmap, ncols, p, (TF*)pg);
  if (e0) cudaEventRecord(e0, st);
  launch_tiles<TF>(variant, grid, st, desc, ntiles, (const TF*)F, (const TF*)pg, (TF*)rowpart, (TF*)colpart, nullptr,
                   status);
  if (e1) cudaEventRecord(e1, st);
  const int gg = std::max(1, std::min((nlam + 255) / 256, 152 * 8));
  gather_tiles_kernel<TF><<<gg, 256, 0, st>>>(P, P.colsub, c0, c1, nlam, (const TF*)rowpart, (const TF*)colpart, q);
}

void launch_gather_lambda(const int* c0, const int* c1, int nlam, const double* qi, double* q, cudaStream_t st) {
  const int gg = std::max(1, std::min((nlam + 255) / 256, 152 * 8));
  gather_lambda_kernel<<<gg, 256, 0, st>>>(c0, c1, nlam, qi, q);
}

void launch_apply(const DevPlan& P, bool fp32, const TileDesc* desc, int ntiles, const void* F, const int* qmap,
                  int64_t ncols, const double* p, void* pg, void* rowpart, void* colpart, const int2* blocks,
                  int nblocks, double* qi, const int* c0, const int* c1, int nlam, double* q, int grid, int variant,
                  int* status, cudaStream_t st, cudaEvent_t ev_tiles0, cudaEvent_t ev_tiles1) {
  if (fp32)
    launch_apply_t<float>(P, desc, ntiles, F, qmap, ncols, p, pg, rowpart, colpart, blocks, nblocks, qi, c0, c1,
                          nlam, q, grid, variant, status, st, ev_tiles0, ev_tiles1);
  else
    launch_apply_t<double>(P, desc, ntiles, F, qmap, ncols, p, pg, rowpart, colpart, blocks, nblocks, qi, c0, c1,
                           nlam, q, grid, variant, status, st, ev_tiles0, ev_tiles1);
}

// The F-streaming part of the apply for the projected CG, whose scatter and
// gather are fused into its vector kernels (the gather sums the tile
// partials itself); skipped when *active == 0 (an iteration enqueued after
// the solve has stopped).
void launch_apply_core(bool fp32, const TileDesc* desc, int ntiles, const void* F, const void* pg, void* rowpart,
                       void* colpart, int grid, int variant, const int* active, int* status, cudaStream_t st,
                       cudaEvent_t ev_tiles0, cudaEvent_t ev_tiles1, bool ev_external) {
  // under stream capture only an external record becomes a timed event-record node
  const unsigned evf = ev_external ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (ev_tiles0) cudaEventRecordWithFlags(ev_tiles0, st, evf);
  if (fp32) {
    launch_tiles<float>(variant, grid, st, desc, ntiles, (const float*)F, (const float*)pg, (float*)rowpart,
                        (float*)colpart, active, status);
    if (ev_tiles1) cudaEventRecordWithFlags(ev_tiles1, st, evf);
  } else {
    launch_tiles<double>(variant, grid, st, desc, ntiles, (const double*)F, (const double*)pg, (double*)rowpart,
                         (double*)colpart, active, status);
    if (ev_tiles1) cudaEventRecordWithFlags(ev_tiles1, st, evf);
  }
}

int apply_variants() { return 6; }

int apply_warps_per_cta(int variant) { return variant < 3 ? kApplyThreads / 32 : kRingW[variant - 3]; }

template <typename TF, int W, int S>
static int occ_ring() {
  const size_t smem = RingCfg<TF>::smem(W, S);
  cudaFuncSetAttribute(apply_ring_kernel<TF, W, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, apply_ring_kernel<TF, W, S>, W * 32, smem);
  return nb;
}

template <typename TF>
static int occ_tiles(int variant) {
  int nb = 0;
  switch (variant) {
    case 0: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, apply_tiles_kernel<TF, 4>, kApplyThreads, 0); break;
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, apply_tiles_kernel<TF, 8>, kApplyThreads, 0); break;
    case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, apply_tiles_kernel<TF, 16>, kApplyThreads, 0); break;
    case 3: nb = occ_ring<TF, 4, 3>(); break;
    case 4: nb = occ_ring<TF, 8, 3>(); break;
    default: nb = occ_ring<TF, 2, 6>(); break;
  }
  return nb;
}

int apply_max_ctas_per_sm(bool fp32, int variant) { return fp32 ? occ_tiles<float>(variant) : occ_tiles<double>(variant); }

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
constexpr int kStaticMaxTiles = kStaticMaxNb * (kStaticMaxNb + 1) / 2;
constexpr int64_t kStaticDoubles = 3 << 19;       // 12 MiB of scratch
// worst case (m = kStaticMaxM, FP64 tiles): gathered p, row and column partials, q_i, 256-byte padding
static_assert((int64_t)kStaticMaxM + 2LL * kStaticMaxTiles * kT + kStaticMaxM + 64 <= kStaticDoubles,
              "static scratch too small for the largest accepted m");
constexpr int kStaticGrid = 152 * 4;

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];
static __device__ __align__(256) TileDesc g_static_desc[kStaticMaxTiles];
static __device__ __align__(256) int2 g_static_blocks[kStaticMaxNb];
static __device__ __align__(256) SubInfo g_static_sub;

namespace {

// Describe the single subdomain, its tile descriptors and blocks in the
// static arrays and zero the padding of the gathered p (every other slot the
// apply reads is overwritten before it is read, so nothing else needs clearing).
template <typename TF>
__global__ void static_setup_kernel(int m, int nb, TF* pg) {
  const int vr = m - kT * (nb - 1);
  if (threadIdx.x == 0) {
    SubInfo S{};
    S.m = m;
    S.m_pad = nb * kT;
    S.nb = nb;
    S.vr = vr;
    S.tpart = 0;
    g_static_sub = S;
  }
  const int ntile = nb * (nb + 1) / 2;
  for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
    int b = 0;
    while ((b + 1) * (b + 2) / 2 <= t) ++b;
    const int bj = t - b * (b + 1) / 2;
    TileDesc d{};
    d.f_ofs = tile_offset<(int)sizeof(TF)>(nb, vr, b, bj);
    d.rows = tile_rows(nb, vr, b);
    d.flags = bj == b ? kTileDiag : 0;
    d.prow = b * kT;
    d.pcol = bj * kT;
    d.slot = t;
    g_static_desc[t] = d;
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
  int2* blocks = nullptr;
  SubInfo* sub = nullptr;
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
    if ((e = cudaGetSymbolAddress((void**)&a.blocks, g_static_blocks)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&a.sub, g_static_sub)) != cudaSuccess) return e;
    g_static_addr[dev] = a;
    g_static_ready[dev] = true;
  }
  out = g_static_addr[dev];
  return cudaSuccess;
}

template <typename TF>
feti_status apply_one_static_t(int m, const TF* F, const int* map, const double* p, double* q, cudaStream_t st) {
  // an error left pending by earlier work on this thread belongs to that work: report it without
  // clearing it (so its owner still sees it), and launch nothing
  if (cudaPeekAtLastError() != cudaSuccess) return FETI_ERR_CUDA;
  const int nb = (m + kT - 1) / kT;
  const int m_pad = nb * kT;
  const int64_t ntile = (int64_t)nb * (nb + 1) / 2;
  // scratch layout: [pg: m_pad TF][row partials: ntile kT TF][column partials: ntile kT TF] | [qi: m_pad double]
  const int64_t n_part = ntile * kT;
  const int64_t qi_ofs = (((int64_t)m_pad + 2 * n_part) * (int64_t)sizeof(TF) + 255) / 256 * 256 / 8;
  if (qi_ofs + m_pad > kStaticDoubles || ntile > kStaticMaxTiles) return FETI_ERR_ARG;
  StaticAddrs a;
  if (static_addresses(a) != cudaSuccess) return FETI_ERR_CUDA;
  TF* pg = reinterpret_cast<TF*>(a.scratch);
  TF* rowpart = pg + m_pad;
  TF* colpart = rowpart + n_part;
  double* qi = a.scratch + qi_ofs;
  static_setup_kernel<TF><<<1, 256, 0, st>>>(m, nb, pg);
  scatter_kernel<TF><<<std::max(1, (m + 255) / 256), 256, 0, st>>>(map, m, p, pg);
  const int wpc = kApplyThreads / 32;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((ntile + wpc - 1) / wpc, kStaticGrid));
  launch_tiles<TF>(0, grid, st, a.desc, (int)ntile, F, pg, rowpart, colpart);
  DevPlan P{};
  P.sub = a.sub;
  launch_reduce<TF>(P, a.blocks, nb, rowpart, colpart, qi, st);
  static_accumulate_kernel<<<std::max(1, (m + 255) / 256), 256, 0, st>>>(map, m, qi, q);
  if (cudaGetLastError() != cudaSuccess) return FETI_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FETI_ERR_CUDA;
  return FETI_OK;
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
