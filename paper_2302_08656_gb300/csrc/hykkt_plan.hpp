// Host-side plan of the saddle-point specialised solve (Sec. V; the method in
// kkt.h): the blocks of K as position lists into K's values, and the pattern
// of H_g = H + J_I^T D_I^{-1} J_I + gamma J_E^T J_E with, per entry, the list
// of its terms in a fixed order.
#pragma once
#include <cstdint>
#include <vector>

namespace kktgb {

// One term of an entry of H_g: k == -1: K value a (an entry of H); k == -2:
// gamma * K_a * K_b (a pair of J_E entries in one equality row); k >= 0:
// K_a * K_b / d_I[k] (a pair of J_I entries in inequality row k).
struct HgTerm {
    int a, b, k;
};

struct HykktPlan {
    int n = 0, np = 0, mE = 0, mI = 0;
    std::vector<int> dpos;                         // position of each dual row's diagonal (mE + mI)
    std::vector<int> je_p, je_c, je_v;             // J_E by rows: CSR pointers, primal columns, positions in K
    std::vector<int> ji_p, ji_c, ji_v;             // J_I by rows
    std::vector<int> jet_p, jet_c, jet_v;          // J_E^T by primal rows: pointers, equality rows, positions
    std::vector<int> jit_p, jit_c, jit_v;          // J_I^T by primal rows
    std::vector<int> hg_p, hg_c;                   // pattern of H_g (np x np, sorted columns, diagonal stored)
    std::vector<int64_t> term_ptr;                 // terms of entry e: term[term_ptr[e] .. term_ptr[e + 1] - 1]
    std::vector<HgTerm> term;                      // in the order: the H entry, J_I pairs by row, J_E pairs by row
};

// Build the plan from K's CSR pattern (n x n, 0-based; unknowns ordered
// primal, m_eq equality duals, inequality duals). Returns 0; 1 if the row
// pointers are not monotone from 0 or an index is out of range; 2 if the
// (2,2) block is not diagonal; 3 if a dual row has no stored diagonal.
int build_hykkt_plan(int n, int n_primal, int m_eq, const int32_t* rowptr, const int32_t* colidx, HykktPlan& p);

}  // namespace kktgb
