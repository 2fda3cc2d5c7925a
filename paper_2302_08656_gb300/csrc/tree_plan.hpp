// Host-side plan of the tree part of the schedule: the top levels of the
// assembly tree that the persistent kernels (tree.cu) refactor and solve.
#pragma once
#include "analysis.hpp"
#include "kernels.cuh"

#include <cstddef>
#include <vector>

namespace kktgb {

constexpr size_t kTreeSmemLimit = 220 * 1024;   // dynamic shared memory of one CTA
constexpr size_t kStageLimit = 96 * 1024;       // largest staged panel / U12 block
constexpr size_t kFwdPanelSmem = 110 * 1024;    // forward chains stage panels only below this (two CTAs per SM)

// Fronts of the levels from `split` up, in level-major order (tree index q),
// their children, factorization units and gather maps; shared-memory sizes
// of the three kernels.
struct TreePlan {
    int split = 0;
    std::vector<TreeFront> fr;
    std::vector<TreeKid> kid;
    std::vector<FrontTile> unit;
    std::vector<FrontTile> unit_fused;  // factor units and, after each level, its forward-solve units (ti = -1)
    std::vector<int> inv;
    // chains of the backward substitution: a chain starts at a root or at a
    // front whose parent has two or more children in the tree part, and
    // continues while the last front has exactly one child in the tree part;
    // chains in descending order of their first front (a chain waits only for
    // the chain that holds its first front's parent, which comes earlier)
    std::vector<int> bwd_chain, bwd_chain_ptr;
    TreeSched ts;
    size_t fac_smem = 0, fwd_smem = 0, bwd_smem = 0;
    int64_t alg_bytes = 0;              // multifrontal traffic of one refactorization of the tree part
    // the tree part's share of the factorization: original entries of K
    // assembled into its fronts, structural entries of L + U in its pivot
    // columns / rows, and its pivots
    int64_t nnz_k = 0, nnz_lu = 0;
    int pivots = 0;
};

// min_fronts: the top levels with fewer fronts than this go to the tree part
// (0: none); es: bytes per factor value.
void build_tree(const Analysis& an, int min_fronts, size_t es, TreePlan& tp);

size_t tree_kid_offset(const TreeSched& t, size_t es);
size_t tree_factor_smem(const TreeSched& t, size_t es);
size_t tree_fwd_smem(const TreeSched& t, size_t es);
size_t tree_bwd_smem(const TreeSched& t, size_t es);

}  // namespace kktgb
