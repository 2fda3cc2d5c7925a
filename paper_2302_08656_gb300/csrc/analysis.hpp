// Host-side analysis of a KKT sparsity pattern (the paper's analysis stage,
// Sec. II: permutations, pivot order and the nonzero pattern of the factors
// are fixed once and reused for every K_k, Alg. 1).
//
// The numeric factorization runs multifrontally over a supernodal assembly
// tree: every supernode s owns a dense F_s x F_s frontal matrix over its row
// set R_s (pivots first, then the rows of its contribution block). All arrays
// here are uploaded once and never change across refactorizations.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace kktgb {

struct Analysis {
    int n = 0;
    int64_t nnz = 0;
    // elimination order (after postordering): perm[k] = original index at step k
    std::vector<int> perm, iperm;
    // supernodes in postorder; pivots of s are steps sn_first[s] .. sn_first[s+1]-1
    int ns = 0;
    std::vector<int> sn_first, sn_parent, sn_front;   // sn_front[s] = F_s
    std::vector<int64_t> rows_ptr;                     // R_s = rows[rows_ptr[s] .. rows_ptr[s+1])
    std::vector<int> rows;                             // step indices, pivots first, ascending
    // children of each supernode, ascending
    std::vector<int> child_ptr, child_list;
    // fronts grouped by level (leaves first)
    std::vector<int> level_ptr, level_fronts;
    int n_levels = 0;
    // original entries assembled into each front: local position a + b*F and CSR index
    std::vector<int64_t> asm_ptr;
    std::vector<int> asm_pos, asm_src;
    // relative indices: CB row t of front s sits at row rel[rel_ptr[s] + t] of its parent front
    std::vector<int64_t> rel_ptr;
    std::vector<int> rel;
    // rel is increasing, so a contribution block's rows that land on pivots of
    // the parent come first: cb_split[s] of them
    std::vector<int> cb_split;
    // factor panel (F*w + w*(F-w) values) and contribution block ((F-w)^2) offsets
    std::vector<int64_t> panel_off, cb_off;
    int64_t panel_total = 0, cb_total = 0;
    // structural entries of L below the diagonal in column (step) j; U row j
    // has the same count plus its diagonal (symmetric structure)
    std::vector<int> colcount;
    // statistics
    int64_t nnz_l = 0, nnz_u = 0;          // structural, diagonal counted in U
    int64_t stored_factor = 0;             // values stored (incl. amalgamation zeros)
    double flops = 0.0;                    // dense front flops actually executed
    double flops_exact = 0.0;              // sum over exact structure
    int max_front = 0, max_pivots = 0;
};

struct AnalysisOptions {
    int ordering = 0;                 // 0 = own minimum degree, 1 = user, 2 = natural
    const int* user_perm = nullptr;   // user_perm[k] = original index eliminated k-th
    int relax_small = 16;             // always merge a chain while the merged front has <= this many pivots and few zeros
    double relax_zeros = 0.15;        // max fraction of explicit zeros added by one merge
    int max_pivots = 64;              // never grow a supernode beyond this many pivots
};

// Returns empty string on success, else an error message. Requires a
// structurally symmetric CSR pattern with sorted, unique column indices and a
// stored diagonal entry in every row.
std::string analyze_pattern(int n, const int* rowptr, const int* colidx,
                            const AnalysisOptions& opt, Analysis& out);

// Sliced ELLPACK copy of a CSR pattern (slices of 32 rows, one row per warp
// lane, entries of a row k = 0, 1, ... at slot off[s] + 32 k + lane, in their
// CSR order). Rows are sorted by length (longest first, then by index) within
// windows of `window` rows before they are cut into slices, so a slice's width
// -- its longest row -- wastes few slots. Fixed for the pattern, like the
// rest of the analysis; the per-refactor copies of K and D K D live in this
// layout so that row sums, row maxima and residuals run one lane per row with
// no cross-lane reduction.
struct SellPlan {
    int nslices = 0;
    int64_t slots = 0;
    std::vector<int64_t> off;         // nslices + 1 slot offsets (width of slice s = (off[s+1]-off[s]) / 32)
    std::vector<int> row;             // nslices * 32: row of each lane, -1 for a lane past the last row
    std::vector<int> ci;              // slots: column index, -1 for padding
    std::vector<int> src;             // slots: CSR position of the entry, -1 for padding
    std::vector<int> csr2sell;        // nnz: slot of each CSR position
};

constexpr int kSellWindow = 4096;

void build_sell(int n, const int* rowptr, const int* colidx, int window, SellPlan& out);

// Quotient-graph minimum-degree ordering (exact external degrees, element
// absorption). order[k] = node eliminated k-th.
void min_degree_quotient(int n, const int* rowptr, const int* colidx, std::vector<int>& order);

}  // namespace kktgb
