// Test driver: runs the library's host analysis and tree plan on a CSR
// pattern read from binary files and writes the plan of the persistent tree
// kernels as raw int64 files, for the ordering checks in
// test_tree_plan_cpu.py.
//   tree_plan_dump <in-prefix> <out-prefix> <max_pivots> <min_fronts>
#include "analysis.hpp"
#include "tree_plan.hpp"

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

static void write_all(const std::string& f, const std::vector<int64_t>& v)
{
    std::ofstream out(f, std::ios::binary);
    out.write(reinterpret_cast<const char*>(v.data()), (std::streamsize)(v.size() * sizeof(int64_t)));
}

int main(int argc, char** argv)
{
    if (argc != 5) { std::fprintf(stderr, "usage: tree_plan_dump <in> <out> <max_pivots> <min_fronts>\n"); return 2; }
    const std::string in = argv[1], out = argv[2];
    const std::vector<int> nv = read_all<int>(in + ".n"), rp = read_all<int>(in + ".rp"), ci = read_all<int>(in + ".ci");
    AnalysisOptions opt;
    opt.max_pivots = std::atoi(argv[3]);
    Analysis a;
    const std::string err = analyze_pattern(nv[0], rp.data(), ci.data(), opt, a);
    if (!err.empty()) { std::fprintf(stderr, "%s\n", err.c_str()); return 1; }
    TreePlan tp;
    build_tree(a, std::atoi(argv[4]), sizeof(double), tp);
    std::vector<int64_t> head = {tp.split, a.n_levels, a.ns, (int64_t)tp.fr.size(), tp.alg_bytes};
    std::vector<int64_t> fr, kid, unit, fused, level(a.ns), sn_parent(a.sn_parent.begin(), a.sn_parent.end());
    for (int l = 0; l < a.n_levels; ++l)
        for (int t = a.level_ptr[l]; t < a.level_ptr[l + 1]; ++t) level[a.level_fronts[t]] = l;
    for (const TreeFront& d : tp.fr) {
        fr.insert(fr.end(), {d.f, d.parent, d.nt, d.units, d.kid_begin, d.kid_end});
    }
    for (const TreeKid& k : tp.kid) kid.push_back(k.q);
    for (const FrontTile& u : tp.unit) unit.insert(unit.end(), {u.front, u.ti, u.tj});
    for (const FrontTile& u : tp.unit_fused) fused.insert(fused.end(), {u.front, u.ti, u.tj});
    std::vector<int64_t> child_ptr(a.child_ptr.begin(), a.child_ptr.end()), child_list(a.child_list.begin(), a.child_list.end());
    write_all(out + ".head", head);
    write_all(out + ".fr", fr);
    write_all(out + ".kid", kid);
    write_all(out + ".unit", unit);
    write_all(out + ".fused", fused);
    write_all(out + ".level", level);
    write_all(out + ".sn_parent", sn_parent);
    write_all(out + ".child_ptr", child_ptr);
    write_all(out + ".child_list", child_list);
    write_all(out + ".asm_ptr", std::vector<int64_t>(a.asm_ptr.begin(), a.asm_ptr.end()));
    write_all(out + ".sn_first", std::vector<int64_t>(a.sn_first.begin(), a.sn_first.end()));
    write_all(out + ".sn_front", std::vector<int64_t>(a.sn_front.begin(), a.sn_front.end()));
    write_all(out + ".bwd_chain", std::vector<int64_t>(tp.bwd_chain.begin(), tp.bwd_chain.end()));
    write_all(out + ".bwd_chain_ptr", std::vector<int64_t>(tp.bwd_chain_ptr.begin(), tp.bwd_chain_ptr.end()));
    return 0;
}
