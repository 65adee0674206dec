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
constexpr int kApplyChunk = 8;  // tiles per apply work item (one tile row is cut into chunks)
constexpr int kApplyWarps = 8;  // consumer warps of the apply; row partials are kept per warp

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
  int64_t trow;      // base of this subdomain's tile-row partials (nb*kT entries) == qcol
  int64_t tpart;     // base of this subdomain's per-tile column partials (ntile*kT entries)
  int64_t rpart;     // base of this subdomain's row partials (nb * ceil(nb / kApplyChunk) * kT entries)
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

// F_i storage: lower tiles (bi, bj), bj <= bi, tile rows kT wide; block row
// bi < nb - 1 holds kT rows per tile, the last block row only S.vr rows.
__host__ __device__ inline int64_t tile_offset(int nb, int vr, int bi, int bj) {
  if (bi < nb - 1) return ((int64_t)bi * (bi + 1) / 2 + bj) * kT * kT;
  return ((int64_t)(nb - 1) * nb / 2) * kT * kT + (int64_t)bj * vr * kT;
}
__host__ __device__ inline int tile_rows(int nb, int vr, int bi) { return bi < nb - 1 ? kT : vr; }
// Position of element (r, c) inside a stored tile: rows of kT values, the
// 16-byte chunks of row r XOR-swizzled by r (so that 8 consecutive rows read
// the same logical chunk from 8 different shared-memory banks).
template <int ESZ>
__host__ __device__ inline int tile_pos(int r, int c) {
  constexpr int cw = 16 / ESZ, nch = kT / cw;
  return r * kT + (((c / cw) ^ (r % nch)) * cw) + (c % cw);
}
__host__ __device__ inline int64_t F_size(int nb, int vr) {
  return nb == 0 ? 0 : ((int64_t)(nb - 1) * nb / 2) * kT * kT + (int64_t)nb * vr * kT;
}

// One F tile of the explicit apply (host-built, 32 bytes).
enum : int { kTileFirst = 1, kTileLast = 2 };
struct __align__(16) TileDesc {
  int64_t f_ofs;   // element offset of the tile in the F storage
  int rows;        // stored rows (kT, or the ragged last block row)
  int flags;       // kTileFirst / kTileLast of its work item
  int prow;        // pg offset of the tile's row block
  int pcol;        // pg offset of the tile's column block
  int col_slot;    // column-partial slot (tile index in the subdomain's partial array + base), -1 on the diagonal
  int row_slot;    // row-partial slot of the work item (written after its last tile)
};

// status word bits written by kernels
enum : int { kStatNotSPD = 1, kStatTimeout = 2, kStatBadPlan = 4 };

}  // namespace feti
