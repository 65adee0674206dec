// Host-side symbolic analysis for the FETI dual-operator path.
//
// Runs once per sparsity pattern (paper Sec. III, symbolic/numeric split and
// Algorithm 2's preparation step): a fill-reducing nested-dissection
// ordering, the elimination tree, supernodes, the multifrontal plan used by
// the numeric Cholesky, and -- per distinct set of B-touched DOFs -- the
// pruned right-hand-side plan (X_i = L_i^{-1} P_i B_i^T column j is zero
// above row s_j) and the SYRK tile lists for F_i = X_i^T X_i.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace feti {

constexpr int kTile = 64;  // F tile edge (apply and SYRK)
// Fronts up to kSmallFront wide whose whole subtree is as small are factored
// by one warp each in shared memory; fronts up to kMidFront wide by the whole
// CTA in shared memory; larger ones by the tiled CTA path.
constexpr int kSmallFront = 40;
constexpr int kMidFront = 112;

// padded row length of a supernode X block (16-byte aligned rows)
inline int xpad(int w) { return (w + 7) & ~7; }

struct PatternPlan {
  int n = 0;
  std::vector<int> perm;   // new -> old DOF
  std::vector<int> iperm;  // old -> new DOF
  int nsn = 0;             // supernodes, in postorder (children before parents)
  std::vector<int> sn_c0, sn_w, sn_r, sn_parent, sn_first_desc;
  std::vector<int64_t> sn_rows_off;  // struct_below rows (new numbering), size nsn+1
  std::vector<int> rows;
  std::vector<int> col2sn;
  std::vector<int> ch_off, ch_list;  // children of each supernode (CSR)
  std::vector<int64_t> rel_off;      // extend-add map of s into its parent, size nsn+1
  std::vector<int> rel;
  std::vector<int64_t> Lofs;         // column-major (w+r) x w panel of each supernode
  int64_t Lsize = 0;
  std::vector<int64_t> kmap_off;     // per supernode, size nsn+1
  std::vector<int> kmap_src;         // CSR index of K entry
  std::vector<int> kmap_dst;         // offset in the subdomain's L storage
  std::vector<int> diag_src;         // CSR index of each diagonal entry (old numbering)
  std::vector<int64_t> upd_stack_ofs;  // where the r x r update block of s lives
  int64_t chol_stack = 0;            // peak stack (doubles)
  std::vector<int> sn_small;         // 1: the supernode and its whole subtree have fronts <= kSmallFront
  std::vector<int64_t> usm_ofs;      // update block slot of a small supernode (own slots, no overlap)
  int64_t usm_size = 0;              // doubles of all small update blocks
  int64_t chol_front = 0;            // max r*r (doubles)
  int max_f = 0, max_w = 0;
  double chol_flops = 0, nnzL = 0;
  // level schedule of the supernodal tree (height from the leaves), small
  // supernodes before large ones inside a level; update-vector offsets
  int nlev = 0;
  std::vector<int> lvl_off, lvl_sn;
  int nlast = 0;  // columns of the forced root supernode (the DOFs ordered last), 0 if none
  std::vector<int64_t> uofs;  // per supernode, offset of its r-vector
  int64_t usize = 0;
  // Cholesky work split (plan_tasks): the supernodal tree cut into tasks at the roots of heavy subtrees;
  // task 0 holds the tree's roots, a task's parent waits for it, and a split root's update block goes to
  // a hand-over slot instead of the CTA stack
  int ntask = 1;
  std::vector<int> sn_task;        // local task of each supernode
  std::vector<int64_t> sn_hoff;    // hand-over slot of a split root (doubles, relative), -1 otherwise
  std::vector<int> task_parent;    // parent task (-1 for task 0)
  std::vector<int> task_nchild;    // child tasks
  std::vector<int> task_height;    // 0 for tasks without child tasks, else 1 + the tallest child
  std::vector<double> task_cost;   // Cholesky flops of the task's own supernodes
  int64_t hsize = 0;               // doubles of all hand-over slots
  std::vector<int> sn_big;         // 1: a front at least big_f wide or an ancestor of one
  bool has_big = false;
  std::vector<int> task_big;       // 1: the task's supernodes are large (the tensor-core Cholesky's)
  std::vector<int> task_nbig;      // large child tasks
};

// Cut the pattern's supernodal tree into Cholesky tasks: a child subtree whose flops exceed `target` becomes
// a task of its own (recursively), so that one large subdomain can be factored by several CTAs.  big_f > 0:
// the fronts at least big_f wide and their ancestors (the tensor-core Cholesky's work) form tasks of their own,
// cut by the same rule, and every other child of that set starts a task.
void plan_tasks(PatternPlan& P, double target, int big_f = 0);

struct BPlan {
  int m = 0, m_pad = 0, nb = 0;
  std::vector<int> colperm;  // sorted column j -> original B row
  std::vector<int> spos;     // sorted column j -> new-numbered DOF
  std::vector<int> jb, je, jo;  // per supernode: J_s = [jb, je), own columns [jo, je)
  std::vector<int> act;      // supernodes with a non-empty J (postorder)
  std::vector<int64_t> Xofs; // per supernode, |J| x wp block (column j holds w values, padded to wp)
  int64_t Xsize = 0;
  std::vector<int64_t> rhs_stack_ofs;
  int64_t rhs_stack = 0, rhs_front = 0;
  std::vector<int> tile_off, tile_sn;  // SYRK contributions per lower kTile tile (bi,bj)
  int nb2 = 0;                         // 128-wide blocks (tensor-core SYRK)
  std::vector<int> t2_off, t2_sn;      // contributions per lower 128 x 128 tile
  double trsm_flops = 0, syrk_flops = 0, syrk_exec_flops = 0;
};

struct SymbolicOptions {
  int leaf_dofs = 16;
  bool use_coords = true;
};

// K pattern: full symmetric CSR (rowptr int64, col int32).  coords: n x 3 or null.
// last (may be null, nlast entries): DOFs ordered last, as one root supernode (every DOF of a node that
// holds one of them goes with it); the other DOFs are ordered by nested dissection before them.  With the
// DOFs that B touches last, the root front assembled from its children is the Schur complement of the
// interior onto them, and X = L^{-1} P B^T is nonzero in the root block only.
void analyse_pattern(int n, const int64_t* rowptr, const int32_t* col, const double* coords,
                     const SymbolicOptions& opt, PatternPlan& out, const int32_t* last = nullptr, int nlast = 0);
// B: m rows, B_dof[r] = local DOF of row r.
void plan_rhs(const PatternPlan& pp, int m, const int32_t* B_dof, BPlan& out);

uint64_t hash_pattern(int n, const int64_t* rowptr, const int32_t* col);
uint64_t hash_ints(const int32_t* a, int64_t n, uint64_t seed);

}  // namespace feti
