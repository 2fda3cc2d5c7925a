// Host-side plan of the tree part (see tree_plan.hpp).
#include "tree_plan.hpp"

#include <algorithm>

namespace kktgb {

static size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

void build_tree(const Analysis& an, int min_fronts, size_t es, TreePlan& tp)
{
    tp = TreePlan();
    int split = an.n_levels;
    if (min_fronts > 0)
        for (int l = an.n_levels - 1; l >= 0; --l) {
            if (an.level_ptr[l + 1] - an.level_ptr[l] >= min_fronts) break;
            split = l;
        }
    // a front with more children than the kernels stage keeps its level (and all below) level-launched
    for (int l = split; l < an.n_levels; ++l)
        for (int t = an.level_ptr[l]; t < an.level_ptr[l + 1]; ++t) {
            int s = an.level_fronts[t];
            if (an.child_ptr[s + 1] - an.child_ptr[s] > kTreeMaxKids) split = l + 1;
        }
    // tree index: level by level; within a level, fronts ordered by the last
    // tree index among their children (stable), so the units that become
    // ready first take the first tickets of their level
    std::vector<int> tq(an.ns, -1);
    std::vector<std::vector<int>> order(an.n_levels);
    int nq = 0;
    for (int l = split; l < an.n_levels; ++l) {
        std::vector<int>& ord = order[l];
        ord.assign(an.level_fronts.begin() + an.level_ptr[l], an.level_fronts.begin() + an.level_ptr[l + 1]);
        if (l > split) {
            std::vector<std::pair<int, int>> key;                 // (last child index, position)
            for (int t = 0; t < (int)ord.size(); ++t) {
                int last = -1;
                for (int c = an.child_ptr[ord[t]]; c < an.child_ptr[ord[t] + 1]; ++c)
                    last = std::max(last, tq[an.child_list[c]]);
                key.emplace_back(last, t);
            }
            std::sort(key.begin(), key.end());
            std::vector<int> sorted;
            for (const auto& k : key) sorted.push_back(ord[k.second]);
            ord.swap(sorted);
        }
        for (int s : ord) tq[s] = nq++;
    }
    tp.split = split;
    tp.fr.resize(nq);
    TreeSched& ts = tp.ts;
    ts.nq = nq;
    for (int l = split; l < an.n_levels; ++l)
        for (int s : order[l]) {
            const int q = tq[s];
            TreeFront& d = tp.fr[q];
            d.f = s;
            d.first = an.sn_first[s];
            d.w = an.sn_first[s + 1] - d.first;
            d.F = an.sn_front[s];
            const int w = d.w, F = d.F, m = F - w;
            d.ts = w < kTile ? 2 * kTile - w : kTile;            // 32 x 32 mini fronts when w <= 16
            d.nt = m > 0 ? (m + d.ts - 1) / d.ts : 1;
            d.units = d.nt * d.nt;
            d.parent = an.sn_parent[s] >= 0 ? tq[an.sn_parent[s]] : -1;
            d.asm_begin = an.asm_ptr[s];
            d.asm_end = an.asm_ptr[s + 1];
            d.panel_off = an.panel_off[s];
            d.cb_off = an.cb_off[s];
            d.rel_ptr = an.rel_ptr[s];
            d.rows_ptr = an.rows_ptr[s];
            d.inv_off = (int64_t)tp.inv.size();
            d.kid_begin = (int)tp.kid.size();
            for (int c = an.child_ptr[s]; c < an.child_ptr[s + 1]; ++c) {
                const int ch = an.child_list[c];
                TreeKid k{};
                k.q = tq[ch];
                k.mc = an.sn_front[ch] - (an.sn_first[ch + 1] - an.sn_first[ch]);
                k.k = an.cb_split[ch];
                k.units = k.q >= 0 ? tp.fr[k.q].units : 0;
                k.cb_off = an.cb_off[ch];
                k.rel_ptr = an.rel_ptr[ch];
                tp.kid.push_back(k);
                const size_t base = tp.inv.size();
                tp.inv.resize(base + m, -1);
                for (int r = 0; r < k.mc; ++r) {
                    const int pos = an.rel[an.rel_ptr[ch] + r];
                    if (pos >= w) tp.inv[base + (pos - w)] = r;
                }
            }
            d.kid_end = (int)tp.kid.size();
            // original entries (value + position + source index), panel, own CB written, children's CB read
            tp.alg_bytes += (d.asm_end - d.asm_begin) * (int64_t)(es + 8) + ((int64_t)F * w + (int64_t)w * m) * (int64_t)es +
                            (int64_t)m * m * (int64_t)es;
            for (int c = d.kid_begin; c < d.kid_end; ++c) tp.alg_bytes += (int64_t)tp.kid[c].mc * tp.kid[c].mc * (int64_t)es;
            tp.nnz_k += d.asm_end - d.asm_begin;
            for (int j = d.first; j < d.first + w; ++j) tp.nnz_lu += 2 * (int64_t)an.colcount[j] + 1;
            tp.pivots += w;
            for (int tj = 0; tj < d.nt; ++tj)
                for (int ti = 0; ti < d.nt; ++ti) tp.unit.push_back(FrontTile{q, ti, tj});
            const int side = w + std::min(d.ts, m);
            ts.m_elems = std::max(ts.m_elems, side * side);
            ts.map_w = std::max(ts.map_w, side);
            ts.max_kids = std::max(ts.max_kids, d.kid_end - d.kid_begin);
            ts.max_F = std::max(ts.max_F, F);
            ts.max_w = std::max(ts.max_w, w);
            ts.max_fw = std::max(ts.max_fw, F * w);
            ts.max_wm = std::max(ts.max_wm, w * m);
        }
    ts.nunits = (int)tp.unit.size();
    // backward chains (see TreePlan)
    {
        std::vector<int> ntk(nq, 0), only(nq, -1);
        for (int q = 0; q < nq; ++q)
            for (int c = tp.fr[q].kid_begin; c < tp.fr[q].kid_end; ++c)
                if (tp.kid[c].q >= 0) {
                    ++ntk[q];
                    only[q] = tp.kid[c].q;
                }
        tp.bwd_chain_ptr.push_back(0);
        for (int q = nq - 1; q >= 0; --q) {
            const int p = tp.fr[q].parent;
            if (p >= 0 && ntk[p] == 1) continue;                  // continues its parent's chain
            for (int x = q;; x = only[x]) {
                tp.bwd_chain.push_back(x);
                if (ntk[x] != 1) break;
            }
            tp.bwd_chain_ptr.push_back((int)tp.bwd_chain.size());
        }
        ts.nchains = (int)tp.bwd_chain_ptr.size() - 1;
    }
    // fused order: level by level, the factorization units of the level, then its forward units
    for (int l = split, u = 0; l < an.n_levels; ++l) {
        const int q0 = tq[order[l].front()];
        const int q1 = q0 + (an.level_ptr[l + 1] - an.level_ptr[l]);
        while (u < (int)tp.unit.size() && tp.unit[u].front < q1) tp.unit_fused.push_back(tp.unit[u++]);
        for (int q = q0; q < q1; ++q) tp.unit_fused.push_back(FrontTile{q, -1, 0});
    }
    ts.nunits_fused = (int)tp.unit_fused.size();
    ts.max_kids = std::max(ts.max_kids, 1);
    ts.fwd_stage = (size_t)ts.max_fw * es <= kStageLimit ? 1 : 0;
    ts.bwd_stage = 2 * (size_t)ts.max_wm * es <= kStageLimit ? 1 : 0;   // two fronts staged at a time
    // forward chains: the children's entries of the largest front's children
    // fit one stage; the two panels are staged if two CTAs per SM still fit
    {
        int most = 1;
        for (const TreeFront& d : tp.fr) {
            int sum = 0;
            for (int c = d.kid_begin; c < d.kid_end; ++c) sum += tp.kid[c].mc;
            most = std::max(most, sum);
        }
        ts.fwd_kstage = std::min(most, kTreeStage);
        ts.fwd_cstage = 1;
        if (tree_fwd_smem(ts, es) > kFwdPanelSmem) ts.fwd_cstage = 0;
    }
    ts.kid_off = tree_kid_offset(ts, es);
    tp.fac_smem = tree_factor_smem(ts, es);
    tp.fwd_smem = tree_fwd_smem(ts, es);
    tp.bwd_smem = tree_bwd_smem(ts, es);
    if (nq > 0 && (tp.fac_smem > kTreeSmemLimit || tp.fwd_smem > kTreeSmemLimit || tp.bwd_smem > kTreeSmemLimit)) {
        TreePlan none;                                            // fronts too large: every level launched
        none.split = an.n_levels;
        tp = none;
    }
}


// factor kernel: mini front and gather maps, or (forward units of the fused
// mode) the forward unit's arrays; the children's descriptors after both
static size_t fwd_arrays(const TreeSched& t, size_t es)
{
    return es * ((size_t)t.max_F + (t.fwd_stage ? (size_t)t.max_fw : (size_t)t.max_w * t.max_w) + kTreeStage) +
           4 * (size_t)kTreeStage;
}

size_t tree_kid_offset(const TreeSched& t, size_t es)
{
    const size_t fac = align16(es * (size_t)t.m_elems) + align16(sizeof(int) * 2 * (size_t)t.max_kids * t.map_w);
    return align16(std::max(fac, fwd_arrays(t, es)));
}

size_t tree_factor_smem(const TreeSched& t, size_t es)
{
    return tree_kid_offset(t, es) + sizeof(TreeKid) * (size_t)t.max_kids;
}

size_t tree_fwd_smem(const TreeSched& t, size_t es)
{
    // v of the current and of the previous front of a chain (max_F each), two
    // staging buffers (own right-hand-side entries, panel or pivot block, the
    // children's values), two buffers of the children's relative indices
    const size_t stage = (size_t)t.max_w + (t.fwd_cstage ? (size_t)t.max_fw : (size_t)t.max_w * t.max_w) + t.fwd_kstage;
    return es * (2 * (size_t)t.max_F + 2 * stage) + 4 * 2 * (size_t)t.fwd_kstage;
}

size_t tree_bwd_smem(const TreeSched& t, size_t es)
{
    // v of the current and of the previous front of a chain (max_F each), then
    // two staging buffers (the current front's and the next one's: own pivot
    // entries, pivot block, staged U12), then two index buffers
    const size_t stage = (size_t)t.max_w + (size_t)t.max_w * t.max_w + (t.bwd_stage ? (size_t)t.max_wm : 0);
    return es * (2 * (size_t)t.max_F + 2 * stage) + 4 * 2 * (size_t)t.max_F;
}

}  // namespace kktgb
