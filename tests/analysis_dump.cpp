// Test driver: runs the library's host analysis on a CSR pattern read from
// binary files and writes every array of the plan as raw int64 little-endian
// files (and the sliced copy of the pattern), for the structural checks in
// test_analysis_cpu.py.
//   analysis_dump <in-prefix> <out-prefix> <max_pivots>
// reads <in>.n (int32 n), <in>.rp (int32 rowptr), <in>.ci (int32 colidx).
#include "analysis.hpp"

#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <string>
#include <vector>

using namespace kktgb;

template <class T>
static std::vector<T> read_all(const std::string& f)
{
    std::ifstream in(f, std::ios::binary | std::ios::ate);
    if (!in) { std::fprintf(stderr, "cannot read %s\n", f.c_str()); std::exit(2); }
    const std::streamsize sz = in.tellg();
    in.seekg(0);
    std::vector<T> v((size_t)sz / sizeof(T));
    in.read(reinterpret_cast<char*>(v.data()), sz);
    return v;
}

template <class V>
static void write_all(const std::string& f, const V& v)
{
    std::vector<int64_t> w(v.begin(), v.end());
    std::ofstream out(f, std::ios::binary);
    out.write(reinterpret_cast<const char*>(w.data()), (std::streamsize)(w.size() * sizeof(int64_t)));
}

int main(int argc, char** argv)
{
    if (argc != 4) { std::fprintf(stderr, "usage: analysis_dump <in> <out> <max_pivots>\n"); return 2; }
    const std::string in = argv[1], out = argv[2];
    const std::vector<int> nv = read_all<int>(in + ".n"), rp = read_all<int>(in + ".rp"), ci = read_all<int>(in + ".ci");
    AnalysisOptions opt;
    opt.max_pivots = std::atoi(argv[3]);
    Analysis a;
    const std::string err = analyze_pattern(nv[0], rp.data(), ci.data(), opt, a);
    if (!err.empty()) { std::fprintf(stderr, "%s\n", err.c_str()); return 1; }
    write_all(out + ".perm", a.perm);
    write_all(out + ".sn_first", a.sn_first);
    write_all(out + ".sn_parent", a.sn_parent);
    write_all(out + ".sn_front", a.sn_front);
    write_all(out + ".rows_ptr", a.rows_ptr);
    write_all(out + ".rows", a.rows);
    write_all(out + ".child_ptr", a.child_ptr);
    write_all(out + ".child_list", a.child_list);
    write_all(out + ".level_ptr", a.level_ptr);
    write_all(out + ".level_fronts", a.level_fronts);
    write_all(out + ".asm_ptr", a.asm_ptr);
    write_all(out + ".asm_pos", a.asm_pos);
    write_all(out + ".asm_src", a.asm_src);
    write_all(out + ".rel_ptr", a.rel_ptr);
    write_all(out + ".rel", a.rel);
    write_all(out + ".cb_split", a.cb_split);
    write_all(out + ".panel_off", a.panel_off);
    write_all(out + ".cb_off", a.cb_off);
    const std::vector<int64_t> stats = {a.ns, a.n_levels, a.nnz_l, a.nnz_u, a.max_front, a.max_pivots,
                                        a.panel_total, a.cb_total};
    write_all(out + ".stats", stats);
    SellPlan sp;
    build_sell(nv[0], rp.data(), ci.data(), kSellWindow, sp);
    write_all(out + ".sell_off", sp.off);
    write_all(out + ".sell_row", sp.row);
    write_all(out + ".sell_ci", sp.ci);
    write_all(out + ".sell_src", sp.src);
    write_all(out + ".csr2sell", sp.csr2sell);
    return 0;
}
