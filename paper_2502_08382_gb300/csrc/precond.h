// Host plan of the lumped preconditioner M = W (sum_i B_i K_i B_i^T) W,
// W = (B B^T)^{-1} (see precond.cpp).
#pragma once
#include <cstdint>
#include <vector>

struct feti_ctx;

namespace feti {

struct LumpedPlan {
  std::vector<int> w_off, w_col;  // W, CSR over multipliers (one dense block per node component)
  std::vector<double> w_val;
  std::vector<int> m_off, m_col;  // M_core pattern, CSR over multipliers
  std::vector<int64_t> c_off;     // per M_core entry: its contributions [c_off[e], c_off[e + 1])
  std::vector<int64_t> c_kidx;    // global K value index of a contribution
  std::vector<double> c_sign;     // sign product of the two B rows
};

void plan_lumped(const feti_ctx* c, LumpedPlan& out);

}  // namespace feti
