// Host-side plan of the saddle-point specialised solve (see hykkt_plan.hpp).
#include "hykkt_plan.hpp"

#include <algorithm>

namespace kktgb {

namespace {

// CSR over the primal rows of the transpose of a dual block given by rows
// (pointers p, primal columns c, positions v; m rows)
void transpose_block(int np, int m, const std::vector<int>& p, const std::vector<int>& c, const std::vector<int>& v,
                     std::vector<int>& tp, std::vector<int>& tc, std::vector<int>& tv)
{
    tp.assign(np + 1, 0);
    for (int j : c) ++tp[j + 1];
    for (int i = 0; i < np; ++i) tp[i + 1] += tp[i];
    tc.resize(c.size());
    tv.resize(c.size());
    std::vector<int> fill(tp.begin(), tp.end() - 1);
    for (int r = 0; r < m; ++r)
        for (int k = p[r]; k < p[r + 1]; ++k) {
            tc[fill[c[k]]] = r;
            tv[fill[c[k]]++] = v[k];
        }
}

}  // namespace

int build_hykkt_plan(int n, int n_primal, int m_eq, const int32_t* rowptr, const int32_t* colidx, HykktPlan& p)
{
    const int np = n_primal, mE = m_eq, mI = n - n_primal - m_eq;
    p = HykktPlan{};
    p.n = n;
    p.np = np;
    p.mE = mE;
    p.mI = mI;
    if (rowptr[0] != 0) return 1;
    for (int i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) return 1;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (colidx[k] < 0 || colidx[k] >= n) return 1;
    }
    // the dual rows: J_E / J_I (primal columns) and the (2,2) diagonal
    p.dpos.assign(mE + mI, -1);
    p.je_p.assign(1, 0);
    p.ji_p.assign(1, 0);
    for (int i = np; i < n; ++i) {
        const bool eq = i < np + mE;
        std::vector<int>& c = eq ? p.je_c : p.ji_c;
        std::vector<int>& v = eq ? p.je_v : p.ji_v;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int j = colidx[k];
            if (j < np) {
                c.push_back(j);
                v.push_back((int)k);
            } else if (j == i) {
                p.dpos[i - np] = (int)k;
            } else {
                return 2;
            }
        }
        (eq ? p.je_p : p.ji_p).push_back((int)c.size());
    }
    for (int k = 0; k < mE + mI; ++k)
        if (p.dpos[k] < 0) return 3;
    transpose_block(np, mE, p.je_p, p.je_c, p.je_v, p.jet_p, p.jet_c, p.jet_v);
    transpose_block(np, mI, p.ji_p, p.ji_c, p.ji_v, p.jit_p, p.jit_c, p.jit_v);
    // H_g row by row: every column it touches with its terms, then the
    // columns sorted
    p.hg_p.assign(1, 0);
    p.term_ptr.assign(1, 0);
    std::vector<int> slot(np, -1), cols, order;
    std::vector<std::vector<HgTerm>> acc;
    for (int i = 0; i < np; ++i) {
        cols.clear();
        acc.clear();
        auto at = [&](int j) -> std::vector<HgTerm>& {
            if (slot[j] < 0) {
                slot[j] = (int)cols.size();
                cols.push_back(j);
                acc.emplace_back();
            }
            return acc[slot[j]];
        };
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (colidx[k] < np) at(colidx[k]).push_back(HgTerm{(int)k, -1, -1});
        at(i);                                                    // the diagonal, stored always
        for (int q = p.jit_p[i]; q < p.jit_p[i + 1]; ++q) {       // inequality rows r holding column i
            const int r = p.jit_c[q], a = p.jit_v[q];
            for (int k = p.ji_p[r]; k < p.ji_p[r + 1]; ++k) at(p.ji_c[k]).push_back(HgTerm{a, p.ji_v[k], r});
        }
        for (int q = p.jet_p[i]; q < p.jet_p[i + 1]; ++q) {       // equality rows r holding column i
            const int r = p.jet_c[q], a = p.jet_v[q];
            for (int k = p.je_p[r]; k < p.je_p[r + 1]; ++k) at(p.je_c[k]).push_back(HgTerm{a, p.je_v[k], -2});
        }
        order.resize(cols.size());
        for (size_t k = 0; k < cols.size(); ++k) order[k] = (int)k;
        std::sort(order.begin(), order.end(), [&](int x, int y) { return cols[x] < cols[y]; });
        for (int k : order) {
            p.hg_c.push_back(cols[k]);
            p.term.insert(p.term.end(), acc[k].begin(), acc[k].end());
            p.term_ptr.push_back((int64_t)p.term.size());
        }
        p.hg_p.push_back((int)p.hg_c.size());
        for (int j : cols) slot[j] = -1;
    }
    return 0;
}

}  // namespace kktgb
