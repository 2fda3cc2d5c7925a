// Host analysis: ordering, elimination tree, symbolic structure, relaxed
// supernodes and the multifrontal schedule. See analysis.hpp.
#include "analysis.hpp"

#include <algorithm>
#include <numeric>
#include <set>
#include <utility>

namespace kktgb {

// ----------------------------------------------------------------- ordering
//
// Minimum degree on the quotient graph: eliminated nodes become "elements"
// (cliques kept implicitly as the list of their variables); an element that
// is adjacent to a newly eliminated pivot is absorbed into it. The degree of a
// variable is its exact external degree |A_i U (union of L_e, e in E_i)| - 1,
// recomputed for the variables of each new element. The next pivot is the
// variable of least degree, the lowest index among equals: a binary heap of
// (degree, index) keys holding every live variable once, its key moved when
// its degree changes. Elements found inside a new element
// are absorbed into it (they add nothing to any union), which leaves every
// degree, and so the order, unchanged.
void min_degree_quotient(int n, const int* rowptr, const int* colidx, std::vector<int>& order)
{
    std::vector<std::vector<int>> av(n), ae(n), le(n);
    std::vector<char> state(n, 0);           // 0 variable, 1 element, 2 absorbed
    std::vector<int> deg(n), mark(n, -1), seen(n, -1), wmark(n, -1), wout(n, 0);
    for (int i = 0; i < n; ++i) {
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (colidx[p] != i) av[i].push_back(colidx[p]);
        deg[i] = (int)av[i].size();
    }
    // indexed binary min-heap of the live variables, keys (degree << 32) | index
    // (unique; the same order as the (degree, index) pairs), hpos[i] = slot of i
    auto key = [](int d, int i) { return ((uint64_t)(uint32_t)d << 32) | (uint32_t)i; };
    std::vector<uint64_t> heap(n);
    std::vector<int> hpos(n);
    int hsize = n;
    for (int i = 0; i < n; ++i) { heap[i] = key(deg[i], i); hpos[i] = i; }
    auto place = [&](int k, uint64_t x) { heap[k] = x; hpos[(int)(uint32_t)x] = k; };
    auto sift_up = [&](int k) {
        const uint64_t x = heap[k];
        while (k > 0) {
            const int up = (k - 1) >> 1;
            if (heap[up] <= x) break;
            place(k, heap[up]);
            k = up;
        }
        place(k, x);
    };
    auto sift_down = [&](int k) {
        const uint64_t x = heap[k];
        while (true) {
            int c = 2 * k + 1;
            if (c >= hsize) break;
            if (c + 1 < hsize && heap[c + 1] < heap[c]) ++c;
            if (x <= heap[c]) break;
            place(k, heap[c]);
            k = c;
        }
        place(k, x);
    };
    for (int k = n / 2 - 1; k >= 0; --k) sift_down(k);
    order.clear();
    order.reserve(n);
    int stamp = 0, stamp2 = 0;
    std::vector<int> lp;
    while (hsize > 0) {
        const int p = (int)(uint32_t)heap[0];
        if (--hsize > 0) { place(0, heap[hsize]); sift_down(0); }
        order.push_back(p);
        // L_p = (A_p U union of absorbed elements' variables) \ {p}
        ++stamp;
        mark[p] = stamp;
        lp.clear();
        for (int v : av[p])
            if (state[v] == 0 && mark[v] != stamp) { mark[v] = stamp; lp.push_back(v); }
        for (int e : ae[p]) {
            if (state[e] != 1) continue;
            for (int v : le[e])
                if (state[v] == 0 && mark[v] != stamp) { mark[v] = stamp; lp.push_back(v); }
            state[e] = 2;
            std::vector<int>().swap(le[e]);
        }
        state[p] = 1;
        std::vector<int>().swap(av[p]);
        std::vector<int>().swap(ae[p]);
        le[p] = lp;
        // update every variable of the new element
        for (int i : lp) {
            // drop absorbed elements, add p
            std::vector<int>& E = ae[i];
            size_t w = 0;
            for (int e : E) if (state[e] == 1) E[w++] = e;
            E.resize(w);
            E.push_back(p);
            // prune variables now covered by element p (and p itself)
            std::vector<int>& A = av[i];
            w = 0;
            for (int v : A) if (state[v] == 0 && mark[v] != stamp) A[w++] = v;
            A.resize(w);
        }
        // exact external degree of each variable i of L_p: every element list
        // of i contains L_p \ {i} (p is one of them), so d_i = |L_p| - 1 plus
        // the variables of A_i and of i's other elements outside L_p, each
        // counted once. First w(e) = |L_e \ L_p| for every other element e
        // next to L_p (one scan per element, dropping dead variables, order
        // kept): an element with w(e) = 0 lies inside L_p and is absorbed into
        // p (every union it took part in is unchanged), and a variable whose
        // only other neighbour is one element e has d_i = |L_p| - 1 + w(e).
        // L_p keeps its marks (stamp); a second stamp array deduplicates per i.
        const int lp_stamp = stamp;
        const int lp_size = (int)lp.size();
        for (int i : lp)
            for (int e : ae[i]) {
                if (e == p || wmark[e] == lp_stamp) continue;
                wmark[e] = lp_stamp;
                std::vector<int>& L = le[e];
                size_t w2 = 0;
                int out = 0;
                for (int v : L) {
                    if (state[v] != 0) continue;
                    L[w2++] = v;
                    if (mark[v] != lp_stamp) ++out;
                }
                L.resize(w2);
                wout[e] = out;
                if (out == 0) {
                    state[e] = 2;
                    std::vector<int>().swap(L);
                }
            }
        for (int i : lp) {
            std::vector<int>& E = ae[i];
            size_t w3 = 0;
            for (int e : E) if (state[e] == 1) E[w3++] = e;
            E.resize(w3);
            int d = lp_size - 1;
            if (av[i].empty() && E.size() == 2) {
                d += wout[E[0] == p ? E[1] : E[0]];
            } else {
                const int st2 = ++stamp2;
                for (int v : av[i])
                    if (state[v] == 0 && mark[v] != lp_stamp && seen[v] != st2) { seen[v] = st2; ++d; }
                for (int e : E) {
                    if (e == p) continue;
                    for (int v : le[e])
                        if (mark[v] != lp_stamp && seen[v] != st2) { seen[v] = st2; ++d; }
                }
            }
            if (d != deg[i]) {
                const int k = hpos[i];
                heap[k] = key(d, i);
                if (d < deg[i]) sift_up(k); else sift_down(k);
                deg[i] = d;
            }
        }
    }
}

// ------------------------------------------------------------------ helpers

static int find_pos(const int* a, int len, int key)
{
    const int* it = std::lower_bound(a, a + len, key);
    if (it == a + len || *it != key) return -1;
    return (int)(it - a);
}

std::string analyze_pattern(int n, const int* rowptr, const int* colidx,
                            const AnalysisOptions& opt, Analysis& out)
{
    if (n <= 0) return "n must be positive";
    if (rowptr[0] != 0) return "rowptr[0] must be 0";
    const int64_t nnz = rowptr[n];
    for (int i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) return "rowptr not monotone";
        bool diag = false;
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int c = colidx[p];
            if (c < 0 || c >= n) return "column index out of range";
            if (p > rowptr[i] && colidx[p - 1] >= c) return "column indices not sorted/unique";
            if (c == i) diag = true;
        }
        if (!diag) return "missing diagonal entry";
    }
    {   // structural symmetry: with sorted rows and column counts equal to the
        // row counts, the pattern is symmetric iff its transpose (rows built
        // in ascending order by a counting sort) has the same column indices
        std::vector<int> cnt(n, 0);
        for (int64_t p = 0; p < nnz; ++p) cnt[colidx[p]]++;
        for (int i = 0; i < n; ++i)
            if (cnt[i] != rowptr[i + 1] - rowptr[i]) return "pattern is not structurally symmetric";
        std::vector<int> tfill(rowptr, rowptr + n), tcol(nnz);
        for (int i = 0; i < n; ++i)
            for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) tcol[tfill[colidx[p]]++] = i;
        if (!std::equal(tcol.begin(), tcol.end(), colidx)) return "pattern is not structurally symmetric";
    }

    // ---- ordering
    std::vector<int> q;
    if (opt.ordering == 1) {
        if (!opt.user_perm) return "user ordering requested without a permutation";
        q.assign(opt.user_perm, opt.user_perm + n);
        std::vector<char> seen(n, 0);
        for (int k = 0; k < n; ++k) {
            if (q[k] < 0 || q[k] >= n || seen[q[k]]) return "user permutation is not a permutation";
            seen[q[k]] = 1;
        }
    } else if (opt.ordering == 2) {
        q.resize(n);
        std::iota(q.begin(), q.end(), 0);
    } else {
        min_degree_quotient(n, rowptr, colidx, q);
    }
    std::vector<int> qinv(n);
    for (int k = 0; k < n; ++k) qinv[q[k]] = k;

    // ---- elimination tree of the permuted pattern (Liu, path compression)
    std::vector<int> parent(n, -1), anc(n, -1);
    for (int k = 0; k < n; ++k) {
        int orig = q[k];
        for (int p = rowptr[orig]; p < rowptr[orig + 1]; ++p) {
            int i = qinv[colidx[p]];
            if (i >= k) continue;
            int r = i;
            while (anc[r] != -1 && anc[r] != k) { int t = anc[r]; anc[r] = k; r = t; }
            if (anc[r] == -1) { anc[r] = k; parent[r] = k; }
        }
    }
    // ---- postorder (children ascending)
    std::vector<int> chead(n, -1), cnext(n, -1);
    for (int k = n - 1; k >= 0; --k)
        if (parent[k] >= 0) { cnext[k] = chead[parent[k]]; chead[parent[k]] = k; }
    std::vector<int> post;
    post.reserve(n);
    {
        std::vector<int> stk;
        for (int r = 0; r < n; ++r) {
            if (parent[r] != -1) continue;
            stk.push_back(r);
            std::vector<int> it;   // iterate children manually
            std::vector<int> cur;
            cur.push_back(chead[r]);
            it.push_back(r);
            while (!it.empty()) {
                int node = it.back();
                int& c = cur.back();
                if (c != -1) {
                    int child = c;
                    c = cnext[c];
                    it.push_back(child);
                    cur.push_back(chead[child]);
                } else {
                    post.push_back(node);
                    it.pop_back();
                    cur.pop_back();
                }
            }
            stk.pop_back();
        }
    }
    std::vector<int> ipost(n);
    for (int t = 0; t < n; ++t) ipost[post[t]] = t;
    out.n = n;
    out.nnz = nnz;
    out.perm.resize(n);
    out.iperm.resize(n);
    for (int t = 0; t < n; ++t) out.perm[t] = q[post[t]];
    for (int t = 0; t < n; ++t) out.iperm[out.perm[t]] = t;
    std::vector<int> par(n, -1);
    for (int t = 0; t < n; ++t) par[t] = parent[post[t]] >= 0 ? ipost[parent[post[t]]] : -1;

    // ---- symbolic structure of every column of L (rows > j, ascending)
    std::vector<std::vector<int>> st(n);
    std::vector<int> nchild(n, 0);
    std::vector<std::vector<int>> kids(n);
    for (int t = 0; t < n; ++t) if (par[t] >= 0) { nchild[par[t]]++; kids[par[t]].push_back(t); }
    {
        std::vector<int> mark(n, -1);
        for (int j = 0; j < n; ++j) {
            std::vector<int>& s = st[j];
            int orig = out.perm[j];
            for (int p = rowptr[orig]; p < rowptr[orig + 1]; ++p) {
                int i = out.iperm[colidx[p]];
                if (i > j && mark[i] != j) { mark[i] = j; s.push_back(i); }
            }
            for (int c : kids[j])
                for (int i : st[c])
                    if (i > j && mark[i] != j) { mark[i] = j; s.push_back(i); }
            std::sort(s.begin(), s.end());
        }
    }
    int64_t nnzl = 0;
    double fl_exact = 0;
    out.colcount.resize(n);
    for (int j = 0; j < n; ++j) {
        int64_t c = (int64_t)st[j].size();
        out.colcount[j] = (int)c;
        nnzl += c;
        fl_exact += (double)c + 2.0 * (double)c * (double)c;   // symmetric structure: |L col| = |U row|
    }
    out.nnz_l = nnzl;
    out.nnz_u = nnzl + n;
    out.flops_exact = fl_exact;

    // ---- fundamental supernodes
    struct SN { int first, last, parent; int64_t F; double zeros; std::vector<int> kids; bool alive; };
    std::vector<SN> sn;
    std::vector<int> sn_of(n, -1);
    for (int j = 0; j < n;) {
        int f = j;
        while (j + 1 < n && par[j] == j + 1 && nchild[j + 1] == 1 && st[j].size() == st[j + 1].size() + 1)
            ++j;
        SN s;
        s.first = f; s.last = j; s.parent = -1;
        s.F = (int64_t)(j - f + 1) + (int64_t)st[j].size();
        s.zeros = 0; s.alive = true;
        for (int t = f; t <= j; ++t) sn_of[t] = (int)sn.size();
        sn.push_back(std::move(s));
        ++j;
    }
    for (size_t s = 0; s < sn.size(); ++s) {
        int pj = par[sn[s].last];
        sn[s].parent = pj >= 0 ? sn_of[pj] : -1;
        if (pj >= 0) sn[sn_of[pj]].kids.push_back((int)s);
    }
    // ---- relaxed amalgamation of the last (contiguous) child into its parent
    auto stored = [](int64_t F, int64_t w) { return (double)(F * w + w * (F - w)); };
    for (size_t p = 0; p < sn.size(); ++p) {
        while (true) {
            SN& P = sn[p];
            int c = -1;
            for (int k : P.kids) if (sn[k].alive && sn[k].last + 1 == P.first) c = k;
            if (c < 0) break;
            SN& Cn = sn[c];
            int64_t wc = Cn.last - Cn.first + 1, wp = P.last - P.first + 1;
            int64_t w = wc + wp, F = wc + P.F;
            if (w > opt.max_pivots) break;
            double newz = 2.0 * (double)wc * (double)(P.F - (Cn.F - wc));
            double z = Cn.zeros + P.zeros + newz;
            double tot = stored(F, w);
            bool ok = (z <= opt.relax_zeros * tot) || (F <= opt.relax_small && w <= opt.relax_small);
            if (!ok) break;
            P.first = Cn.first;
            P.F = F;
            P.zeros = z;
            std::vector<int> nk;
            for (int k : P.kids) if (k != c) nk.push_back(k);
            for (int k : Cn.kids) { nk.push_back(k); sn[k].parent = (int)p; }
            P.kids.swap(nk);
            Cn.alive = false;
        }
    }
    // ---- split supernodes with more than max_pivots pivots into a chain of
    // pieces. The last column of every supernode is an elimination-tree
    // ancestor of all its columns, so a piece's contribution rows are rows of
    // the next piece and the split needs no new structure.
    std::vector<std::pair<int, int>> ranges;   // (first, last) in column order
    for (size_t k = 0; k < sn.size(); ++k)
        if (sn[k].alive) ranges.push_back({sn[k].first, sn[k].last});
    std::sort(ranges.begin(), ranges.end());
    {
        std::vector<std::pair<int, int>> split;
        const int cap = std::max(1, opt.max_pivots);
        for (const auto& r : ranges) {
            for (int f = r.first; f <= r.second; f += cap)
                split.push_back({f, std::min(r.second, f + cap - 1)});
        }
        ranges.swap(split);
    }
    const int ns = (int)ranges.size();
    out.ns = ns;
    out.sn_first.assign(ns + 1, n);
    out.sn_parent.assign(ns, -1);
    out.sn_front.assign(ns, 0);
    for (int k = 0; k < ns; ++k) {
        out.sn_first[k] = ranges[k].first;
        for (int j = ranges[k].first; j <= ranges[k].second; ++j) sn_of[j] = k;
    }
    for (int k = 0; k < ns; ++k) {
        int pj = par[ranges[k].second];
        out.sn_parent[k] = pj >= 0 ? sn_of[pj] : -1;
    }
    // row sets: pivots, then the union of the pivot columns' structures below the last pivot
    out.rows_ptr.assign(ns + 1, 0);
    out.rows.clear();
    {
        std::vector<int> mark(n, -1), buf;
        for (int k = 0; k < ns; ++k) {
            int f = out.sn_first[k], l = out.sn_first[k + 1] - 1;
            buf.clear();
            for (int j = f; j <= l; ++j)
                for (int i : st[j])
                    if (i > l && mark[i] != k) { mark[i] = k; buf.push_back(i); }
            std::sort(buf.begin(), buf.end());
            for (int j = f; j <= l; ++j) out.rows.push_back(j);
            out.rows.insert(out.rows.end(), buf.begin(), buf.end());
            out.rows_ptr[k + 1] = (int64_t)out.rows.size();
            out.sn_front[k] = (int)(out.rows_ptr[k + 1] - out.rows_ptr[k]);
        }
    }
    // children lists and levels
    out.child_ptr.assign(ns + 1, 0);
    for (int k = 0; k < ns; ++k) if (out.sn_parent[k] >= 0) out.child_ptr[out.sn_parent[k] + 1]++;
    for (int k = 0; k < ns; ++k) out.child_ptr[k + 1] += out.child_ptr[k];
    out.child_list.assign(out.child_ptr[ns], 0);
    {
        std::vector<int> fill(out.child_ptr.begin(), out.child_ptr.end() - 1);
        for (int k = 0; k < ns; ++k)
            if (out.sn_parent[k] >= 0) out.child_list[fill[out.sn_parent[k]]++] = k;
    }
    std::vector<int> lev(ns, 0);
    int nlev = 0;
    for (int k = 0; k < ns; ++k) {           // children precede parents
        if (out.sn_parent[k] >= 0) lev[out.sn_parent[k]] = std::max(lev[out.sn_parent[k]], lev[k] + 1);
        nlev = std::max(nlev, lev[k] + 1);
    }
    out.n_levels = nlev;
    out.level_ptr.assign(nlev + 1, 0);
    for (int k = 0; k < ns; ++k) out.level_ptr[lev[k] + 1]++;
    for (int l = 0; l < nlev; ++l) out.level_ptr[l + 1] += out.level_ptr[l];
    out.level_fronts.assign(ns, 0);
    {
        std::vector<int> fill(out.level_ptr.begin(), out.level_ptr.end() - 1);
        for (int k = 0; k < ns; ++k) out.level_fronts[fill[lev[k]]++] = k;
    }
    // supernode of each step
    std::vector<int> snk(n);
    for (int k = 0; k < ns; ++k)
        for (int j = out.sn_first[k]; j < out.sn_first[k + 1]; ++j) snk[j] = k;
    // assembly of original entries: entry (r, c) goes to the front of min(r, c)
    {
        std::vector<int64_t> cnt(ns + 1, 0);
        for (int i = 0; i < n; ++i)
            for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                int r = out.iperm[i], c = out.iperm[colidx[p]];
                cnt[snk[std::min(r, c)] + 1]++;
            }
        for (int k = 0; k < ns; ++k) cnt[k + 1] += cnt[k];
        out.asm_ptr = cnt;
        out.asm_pos.assign(nnz, 0);
        out.asm_src.assign(nnz, 0);
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
        std::vector<int> er(nnz), ec(nnz);              // permuted (row, column) of each slot
        for (int i = 0; i < n; ++i)
            for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                int r = out.iperm[i], c = out.iperm[colidx[p]];
                int64_t at = fill[snk[std::min(r, c)]]++;
                er[at] = r;
                ec[at] = c;
                out.asm_src[at] = p;
            }
        // local positions through a row -> (front, position) map, one front at a time
        std::vector<int> where(n, -1), owner(n, -1);
        for (int k = 0; k < ns; ++k) {
            const int* R = out.rows.data() + out.rows_ptr[k];
            const int F = out.sn_front[k];
            for (int t = 0; t < F; ++t) { where[R[t]] = t; owner[R[t]] = k; }
            for (int64_t at = out.asm_ptr[k]; at < out.asm_ptr[k + 1]; ++at) {
                const int r = er[at], c = ec[at];
                if (owner[r] != k || owner[c] != k) return "internal: entry outside its front";
                out.asm_pos[at] = where[r] + where[c] * F;
            }
        }
    }
    // relative indices of each contribution block in its parent
    out.rel_ptr.assign(ns + 1, 0);
    for (int k = 0; k < ns; ++k) {
        int w = out.sn_first[k + 1] - out.sn_first[k];
        out.rel_ptr[k + 1] = out.rel_ptr[k] + (out.sn_front[k] - w);
    }
    out.rel.assign(out.rel_ptr[ns], 0);
    out.cb_split.assign(ns, 0);
    for (int k = 0; k < ns; ++k) {
        int w = out.sn_first[k + 1] - out.sn_first[k];
        int F = out.sn_front[k];
        int pk = out.sn_parent[k];
        if (F == w) continue;
        if (pk < 0) return "internal: root front with a contribution block";
        const int* R = out.rows.data() + out.rows_ptr[k];
        const int* Rp = out.rows.data() + out.rows_ptr[pk];
        for (int t = w; t < F; ++t) {
            int pos = find_pos(Rp, out.sn_front[pk], R[t]);
            if (pos < 0) return "internal: contribution row missing from the parent front";
            out.rel[out.rel_ptr[k] + (t - w)] = pos;
            if (pos < out.sn_first[pk + 1] - out.sn_first[pk]) out.cb_split[k] = t - w + 1;
        }
    }
    // storage and statistics
    out.panel_off.assign(ns + 1, 0);
    out.cb_off.assign(ns + 1, 0);
    double fl = 0;
    out.max_front = 0;
    out.max_pivots = 0;
    for (int k = 0; k < ns; ++k) {
        int64_t w = out.sn_first[k + 1] - out.sn_first[k], F = out.sn_front[k];
        out.panel_off[k + 1] = out.panel_off[k] + F * w + w * (F - w);
        out.cb_off[k + 1] = out.cb_off[k] + (F - w) * (F - w);
        for (int64_t p = 0; p < w; ++p) fl += (double)(F - p - 1) + 2.0 * (double)(F - p - 1) * (double)(F - p - 1);
        out.max_front = std::max<int>(out.max_front, (int)F);
        out.max_pivots = std::max<int>(out.max_pivots, (int)w);
    }
    out.panel_total = out.panel_off[ns];
    out.cb_total = out.cb_off[ns];
    out.stored_factor = out.panel_total;
    out.flops = fl;
    return std::string();
}

void build_sell(int n, const int* rowptr, const int* colidx, int window, SellPlan& out)
{
    const int64_t nnz = rowptr[n];
    out.nslices = (n + 31) / 32;
    out.off.assign(out.nslices + 1, 0);
    out.row.assign((size_t)out.nslices * 32, -1);
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int w0 = 0; w0 < n; w0 += window) {
        const int w1 = std::min(n, w0 + window);
        std::stable_sort(order.begin() + w0, order.begin() + w1, [&](int a, int b) {
            return rowptr[a + 1] - rowptr[a] > rowptr[b + 1] - rowptr[b];
        });
    }
    for (int s = 0; s < out.nslices; ++s) {
        int width = 0;
        for (int l = 0; l < 32 && s * 32 + l < n; ++l) {
            const int r = order[s * 32 + l];
            out.row[(size_t)s * 32 + l] = r;
            width = std::max(width, rowptr[r + 1] - rowptr[r]);
        }
        out.off[s + 1] = out.off[s] + 32 * (int64_t)width;
    }
    out.slots = out.off[out.nslices];
    out.ci.assign(out.slots, -1);
    out.src.assign(out.slots, -1);
    out.csr2sell.assign(nnz, -1);
    for (int s = 0; s < out.nslices; ++s)
        for (int l = 0; l < 32; ++l) {
            const int r = out.row[(size_t)s * 32 + l];
            if (r < 0) continue;
            for (int p = rowptr[r], k = 0; p < rowptr[r + 1]; ++p, ++k) {
                const int64_t slot = out.off[s] + 32 * (int64_t)k + l;
                out.ci[slot] = colidx[p];
                out.src[slot] = p;
                out.csr2sell[p] = (int)slot;
            }
        }
}

}  // namespace kktgb
