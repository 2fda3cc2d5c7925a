// Test driver: runs the host plan of the saddle-point specialised solve on a
// CSR pattern read from binary files and writes the blocks, the pattern of
// H_g and its term lists as raw int64 files, for test_hykkt_plan_cpu.py.
//   hykkt_plan_dump <in-prefix> <out-prefix> <n_primal> <m_eq>
// Exit status: the plan's return code (0, or 1 / 2 / 3 for a rejected pattern).
#include "hykkt_plan.hpp"

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
    if (!in) { std::fprintf(stderr, "cannot read %s\n", f.c_str()); std::exit(9); }
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
    if (argc != 5) { std::fprintf(stderr, "usage: hykkt_plan_dump <in> <out> <n_primal> <m_eq>\n"); return 9; }
    const std::string in = argv[1], out = argv[2];
    const std::vector<int> nv = read_all<int>(in + ".n"), rp = read_all<int>(in + ".rp"), ci = read_all<int>(in + ".ci");
    HykktPlan p;
    const int st = build_hykkt_plan(nv[0], std::atoi(argv[3]), std::atoi(argv[4]), rp.data(), ci.data(), p);
    if (st != 0) return st;
    write_all(out + ".dpos", p.dpos);
    write_all(out + ".je_p", p.je_p);
    write_all(out + ".je_c", p.je_c);
    write_all(out + ".je_v", p.je_v);
    write_all(out + ".ji_p", p.ji_p);
    write_all(out + ".ji_c", p.ji_c);
    write_all(out + ".ji_v", p.ji_v);
    write_all(out + ".jet_p", p.jet_p);
    write_all(out + ".jet_c", p.jet_c);
    write_all(out + ".jet_v", p.jet_v);
    write_all(out + ".jit_p", p.jit_p);
    write_all(out + ".jit_c", p.jit_c);
    write_all(out + ".jit_v", p.jit_v);
    write_all(out + ".hg_p", p.hg_p);
    write_all(out + ".hg_c", p.hg_c);
    write_all(out + ".term_ptr", p.term_ptr);
    std::vector<int64_t> t;
    t.reserve(3 * p.term.size());
    for (const HgTerm& x : p.term) t.insert(t.end(), {x.a, x.b, x.k});
    write_all(out + ".term", t);
    return 0;
}
