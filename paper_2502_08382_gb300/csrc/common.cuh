// Device-side plan layout shared by the FETI kernels.
//
// The host symbolic phase (symbolic.cpp) produces one plan per distinct K
// pattern and one pruned-RHS plan per distinct set of B-touched DOFs; they
// are concatenated into flat device arrays.  Offsets stored in the tables
// below are absolute within those flat arrays unless marked "relative".
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace feti {

constexpr int kT = 64;          // F tile edge
constexpr int kThreads = 256;   // CTA size of the dense kernels
constexpr int kNB = 32;         // panel block of the dense factorisation / solve

struct SubInfo {
  int n, m, m_pad, nb, nsn, nact, d, nfix;
  int sn0;           // pattern supernode base (sn_* arrays)
  int bsn0;          // bplan supernode base (jb/je/jo/Xofs/rhs_stack_ofs)
  int act0;          // bplan active-list base
  int col0;          // bplan sorted-column base (spos)
  int tile0;         // bplan tile_off base
  int fix0;          // fix arrays base
  int alpha0;        // offset of this subdomain's alpha block
  int t20;           // bplan t2_off base (128 x 128 tiles)
  int nb2;           // 128-wide blocks
  int vr;            // rows of the last block row (m - kT (nb - 1)); that row stores only these
  int nlev;          // levels of the supernodal tree
  int lvl0;          // pattern level-offset base (lvl_off, nlev + 1 entries)
  int64_t kmapb;     // base of this pattern's kmap entries (kmap_off values are absolute)
  int64_t diag0;     // diag_src base
  int64_t Kval;      // subdomain K values base
  int64_t L;         // subdomain L base (doubles)
  int64_t X;         // subdomain X base (elements)
  int64_t F;         // subdomain F tiles base (elements)
  int64_t qcol;      // subdomain sorted-column arrays base (m_pad entries)
  int64_t dof;       // subdomain DOF-vector base (n entries)
  int64_t R;         // subdomain R base (n*d, column-major)
  int64_t trow;      // == qcol (unused)
  int64_t tpart;     // first apply tile of this subdomain times kT (its row / column partial slots)
  int64_t rpart;     // unused
  int64_t hbase;     // base of this subdomain's Cholesky hand-over slots (doubles)
  int64_t lh;        // base of this subdomain's row-major bf16 hi/lo panels (LH, elements)
  int64_t di;        // base of this subdomain's inverted 32 x 32 diagonal blocks of the large panels (DI, floats)
};

struct DevPlan {
  const SubInfo* sub;
  // pattern tables
  const int* sn_c0;
  const int* sn_w;
  const int* sn_r;
  const int* sn_parent;
  const int64_t* sn_rows;    // [sn] absolute offset of struct-below rows (size nsn+1 per pattern)
  const int* rows;
  const int* ch_off;         // [sn] absolute offsets into ch_list (size nsn+1 per pattern)
  const int* ch_list;        // local supernode ids
  const int64_t* rel_off;    // [sn] absolute offsets into rel (size nsn+1 per pattern)
  const int* rel;
  const int64_t* Lofs;       // [sn] relative to the subdomain's L base
  const int64_t* kmap_off;   // [sn] absolute (size nsn+1 per pattern)
  const int* kmap_src;       // relative to the subdomain's K values
  const int* kmap_dst;       // relative to the subdomain's L base
  const int* diag_src;       // relative to the subdomain's K values
  const int64_t* upd_ofs;    // [sn] relative to the CTA stack
  const int* lvl_off;        // [lvl0 + l] absolute offsets into lvl_sn
  const int* lvl_sn;         // local supernode ids, level by level
  const int64_t* uofs;       // [sn] update-vector offset of the supernode (relative to the CTA workspace)
  const int* sn_small;       // [sn] 1: small-subtree supernode (warp-factored front)
  const int64_t* usm_ofs;    // [sn] update-block slot of a small supernode (relative to the CTA's small region)
  const int* sn_task;        // [sn] Cholesky task of the supernode (local to the pattern's split)
  const int64_t* sn_hoff;    // [sn] hand-over slot of a split root (relative to the subdomain's hbase), -1 if none
  const int* task_nchild;    // [global task] child tasks to wait for
  const int* sn_big;         // [sn] 1: factored by the tensor-core Cholesky kernel (large front or ancestor)
  const int* task_nbig;      // [global task] large child tasks (the tensor-core kernel waits for them)
  const int64_t* lh_ofs;     // [sn] offset of the supernode's row-major hi/lo panel in LH (relative to the
                             // subdomain's lh), -1 for fronts the large-front TRSM does not take
  uint16_t* LH;              // row-major bf16 hi/lo copies of the large panels (mixed precision)
  const int64_t* di_ofs;     // [sn] offset of the supernode's inverted diagonal blocks in DI (relative to the
                             // subdomain's di; 4 blocks of 32 x 32 per 128 own rows), -1 where lh_ofs is -1
  float* DI;                 // inverses of the 32 x 32 diagonal blocks of the large panels (FP32)
  double* dinv;              // [dof + j] reciprocal pivots 1 / L_jj (written after the factorisation)
  // bplan tables
  const int* jb;
  const int* je;
  const int* jo;
  const int64_t* Xofs;       // [bsn] relative to the subdomain's X base
  const int64_t* rhs_ofs;    // [bsn] relative to the CTA stack
  const int* act;            // local supernode ids
  const int* spos;           // [col0 + j] new-numbered DOF of sorted column j
  const int* tile_off;       // [tile0 + t] absolute offsets into tile_sn
  const int* tile_sn;        // local supernode ids
  const int* t2_off;         // [t20 + t] absolute offsets into t2_sn (128 x 128 tiles)
  const int* t2_sn;
  // per subdomain
  const int* qmap;           // [qcol + j] global multiplier of sorted column j, -1 for padding
  const int* colsub;         // [qcol + j] subdomain of sorted column j
  const double* qsign;       // [qcol + j] sign of B in sorted column j (0 for padding)
  const int* iperm;          // [diag0 + old DOF] new-numbered DOF (pattern)
  const int* qdof;           // [qcol + j] original local DOF of sorted column j
  const int* colperm;        // [qcol + j] B row of sorted column j
  const int* fix_sn;         // [fix0 + k] supernode holding fixing DOF k
  const int64_t* fix_pos;    // [fix0 + k] diagonal position in L (relative)
  // values
  const double* Kval;
  double* L;
  double* rho;               // [nsub]
};

// F_i storage: lower tiles (bi, bj), bj <= bi, in the order bi (bi + 1) / 2 + bj.
// Off-diagonal tiles are row-major kT x kT; block row bi < nb - 1 holds kT
// rows per tile, the last block row only S.vr rows.  A diagonal tile keeps, for
// each row r, only the 16-byte chunks up to and including the one that holds
// column r (ceil((r + 1) / V) chunks of V = 16 / ESZ values), rows packed back
// to back; the entries right of the diagonal inside that last chunk are zero.
// Every tile and every row of a diagonal tile starts on a 16-byte boundary.
template <int ESZ>
__host__ __device__ inline int64_t diag_row_off(int r) {
  constexpr int V = 16 / ESZ;
  const int64_t q = r / V;
  return (int64_t)V * ((int64_t)V * q * (q + 1) / 2 + (int64_t)(r - V * q) * (q + 1));
}
template <int ESZ>
__host__ __device__ inline int64_t tile_offset(int nb, int vr, int bi, int bj) {
  const int64_t dk = diag_row_off<ESZ>(kT);
  if (bi < nb - 1) return (int64_t)kT * kT * bi * (bi - 1) / 2 + (int64_t)bi * dk + (int64_t)bj * kT * kT;
  const int64_t base = (int64_t)kT * kT * (nb - 1) * (nb - 2) / 2 + (int64_t)(nb - 1) * dk;
  return base + (int64_t)bj * vr * kT;
}
__host__ __device__ inline int tile_rows(int nb, int vr, int bi) { return bi < nb - 1 ? kT : vr; }
// element (r, c) of an off-diagonal tile / of a diagonal tile (c < V ceil((r + 1) / V))
__host__ __device__ inline int tile_pos(int r, int c) { return r * kT + c; }
template <int ESZ>
__host__ __device__ inline int64_t diag_pos(int r, int c) { return diag_row_off<ESZ>(r) + c; }
template <int ESZ>
__host__ __device__ inline int64_t F_size(int nb, int vr) {
  return nb == 0 ? 0 : tile_offset<ESZ>(nb, vr, nb - 1, nb - 1) + diag_row_off<ESZ>(vr);
}
__host__ __device__ inline int64_t F_size_esz(int esz, int nb, int vr) {
  return esz == 4 ? F_size<4>(nb, vr) : F_size<8>(nb, vr);
}

// One F tile of the explicit apply (host-built, 32 bytes).  The tile owns
// row-partial slot `slot` and column-partial slot `slot` (its position in
// the subdomain-major tile order); the descriptor list itself may be in any
// order (largest tiles first, so that the warps' last tiles are small).
enum : int { kTileDiag = 1 };
struct __align__(16) TileDesc {
  int64_t f_ofs;   // element offset of the tile in the F storage
  int rows;        // stored rows (kT, or the ragged last block row)
  int flags;       // kTileDiag for a diagonal tile
  int prow;        // pg offset of the tile's row block
  int pcol;        // pg offset of the tile's column block
  int slot;        // partial slot
  int pad;
};

// (F_i p_i)[j] for column j of a subdomain whose tile partials start at tile
// slot tb (nb blocks): the row partials of the tiles of its block row and the
// column partials of the tiles of its block column, summed in a fixed order
// (bj = 0..b, then bi = b..nb-1) in the precision of the partials (FP64
// conversion and addition run on a narrow pipe of this GPU; FP32 partials
// are summed in FP32).  The loads are issued eight at a time so that they
// overlap; the additions keep that order.
template <typename TF>
__device__ __forceinline__ double colsum_at(int64_t tb, int nb, int j, const TF* rowpart, const TF* colpart) {
  const int b = j / kT, x = j % kT;
  const int nt = nb + 1;  // b + 1 row partials, nb - b column partials
  const int64_t r0 = tb + (int64_t)b * (b + 1) / 2;
  TF s = (TF)0;
  for (int k0 = 0; k0 < nt; k0 += 8) {
    TF v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = k0 + u;
      v[u] = (TF)0;
      if (k <= b) v[u] = rowpart[(r0 + k) * kT + x];
      else if (k < nt) {
        const int bi = k - 1;  // b .. nb - 1
        v[u] = colpart[(tb + (int64_t)bi * (bi + 1) / 2 + b) * kT + x];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k0 + u < nt) s += v[u];
  }
  return (double)s;
}

// colsum_at for sorted column g of subdomain `sub`
template <typename TF>
__device__ __forceinline__ double tile_colsum(const SubInfo& S, int64_t g, const TF* rowpart, const TF* colpart) {
  return colsum_at(S.tpart / kT, S.nb, (int)(g - S.qcol), rowpart, colpart);
}

// Control block of the projected CG (Algorithm 1), in device memory.  The
// vector kernels read and update it; the host reads it once per chunk of
// enqueued iterations.
struct PcgCtrl {
  double wy;      // w.w of the current iterate (M = I: y = w)
  double wy_prev; // w.w before the last iteration's update (a residual replacement divides by it)
  double pq;      // p.q of the current iteration
  double delta;   // step length (w.w) / (p.q)
  double beta;    // (w_new.w_new) / (w.w) for p <- w + beta p
  double wyn;     // w.w after the update
  double nw;      // ||w|| after the update
  double nw0;     // ||w_0||
  double tol;     // relative tolerance on ||w|| / ||w_0||
  double floor;   // rounding level of the residual: 64 eps (||d|| + ||F lambda_0||)
  double rel;     // ||w|| / ||w_0||
  double dd, qq;  // ||d||^2 and ||F lambda_0||^2 (for the floor)
  int active;     // 1 while iterating; kernels of later iterations return when 0
  int it;         // iterations done
  int maxit;
  int conv;       // the last ||w|| met the stopping rule
  int breakdown;  // p.q <= 0 was met
  int restart;    // 1: a residual replacement restarts the search direction (beta = 0)
  int cnt_dot, cnt_upd, cnt_proj;  // arrival counters of the last-block reductions
};
constexpr int kPcgMaxBlocks = 1184;  // block partials per reduction

// One subdomain of a batch of the FP64 adjoint (kern_adjoint.cu).  Offsets in
// doubles into the batch's work buffer (v_ofs: n x 2 m_pad row-major V,
// ws_ofs: m_pad x m_pad sorted W), into W (w_src) and into the element arrays.
struct AdjBatch {
  int sub, m, m_pad, edofs, nelem;
  int zonly;  // 1: V holds only D^{-2} X_u (row length m_pad), for the TRSM-path assembly of F_i
  int64_t qcol, w_src, ws_ofs, v_ofs, el_dofs, el_dk, el_out, dk_stride;
};
constexpr int kBuildCols = 512;  // columns of V_Y per item of the adjoint's X_u W product

// flags of the numeric Cholesky (kern_factor.cu)
enum : int { kCholNoReg = 1, kCholStopRoot = 2, kCholSkipBig = 4 };

// status word bits written by kernels
enum : int { kStatNotSPD = 1, kStatTimeout = 2, kStatBadPlan = 4 };

}  // namespace feti
