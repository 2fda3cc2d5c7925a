// Runtime and C ABI (include/kkt.h): context, device memory pool, launch
// schedule per assembly-tree level, FGMRES refinement driver.
#include "../../include/kkt.h"
#include "analysis.hpp"
#include "kernels.cuh"
#include "tree_plan.hpp"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <vector>

namespace kktgb {
cudaError_t configure_kernels();
}

using namespace kktgb;

namespace {

struct LevelGroup {
    int warp_off = 0, warp_cnt = 0;           // offsets into the device front-id array
    int cta_off = 0, cta_cnt = 0, cta_maxF = 0;
    int panel_off = 0, panel_cnt = 0, panel_maxW = 0;
    int small_maxF = 0, small_maxW = 0, big_maxF = 0, big_maxW = 0;   // solve: warp / CTA classes
    int warp_stage_v = 0, warp_stage_r = 0;   // warp kernel: children's staging per warp (values, indices)
    // refactorization only: childless fronts with F <= 8 / F <= 16 (several per
    // warp), then the rest of the warp class (the solves take the whole class)
    int leaf8_off = 0, leaf8_cnt = 0, leaf16_off = 0, leaf16_cnt = 0;
    int wfac_off = 0, wfac_cnt = 0, wfac_maxF = 0;
    size_t panel_smem = 0;                    // 0 with panel_global = true
    bool panel_global = false;
    int tile_off = 0, tile_cnt = 0;
    int all_off = 0, all_cnt = 0, all_maxF = 0, all_maxW = 0;   // every front of the level (solve)
};

// Device pool: one allocation carved into aligned pieces.
struct Pool {
    char* base = nullptr;
    size_t size = 0, used = 0;
    template <typename X>
    X* take(size_t count)
    {
        size_t bytes = ((count * sizeof(X)) + 255) & ~size_t(255);
        X* p = reinterpret_cast<X*>(base + used);
        used += bytes;
        return p;
    }
};

constexpr int kMaxRestart = 64;
constexpr size_t kRedScratch = 128 + 304 * (kMaxRestart + 2) + 16;
// FGMRES state on the device: Hessenberg matrix ((m + 1) x m, leading
// dimension kMaxRestart + 1), rotations, right-hand side, solution, scale,
// convergence flags
constexpr int kGmLd = kMaxRestart + 1;
constexpr size_t kGmH = 0, kGmCs = kGmH + (size_t)kGmLd * kMaxRestart, kGmSn = kGmCs + kMaxRestart,
                 kGmG = kGmSn + kMaxRestart, kGmY = kGmG + kMaxRestart + 8, kGmScale = kGmY + kMaxRestart + 8,
                 kGmFlag = kGmScale + 8, kGmSize = kGmFlag + kMaxRestart + 8;

}  // namespace

struct kkt_ctx {
    kkt_options opt;
    Analysis an;
    int n = 0, n_primal = 0;
    int batch = 1;                   // numeric instances sharing this analysis
    int64_t nnz = 0;
    int64_t slots = 0;               // sliced copy of K (SellPlan): slots per instance
    std::vector<LevelGroup> levels;
    int64_t scratch_stride = 0;      // panel scratch per CTA (global fallback)
    int max_panel_global = 0;
    Pool pool;
    DevSched sched;
    DevStat* stat = nullptr;
    // numeric buffers (one precision is used)
    DevNum<double> nd;
    DevNum<float> nf;
    double* d_a = nullptr;           // Ruiz buffers
    double* d_b = nullptr;
    double* d_final = nullptr;
    void* panel_scratch = nullptr;
    int* fronts_dev = nullptr;
    FrontTile* tiles_dev = nullptr;
    // persistent kernels of the tree part
    TreeSched tsched;
    int tree_split = 0;
    int64_t tree_bytes = 0;
    int64_t tree_nnz_k = 0, tree_nnz_lu = 0;
    int tree_pivots = 0;
    size_t tf_smem = 0, tfw_smem = 0, tbw_smem = 0;
    int tf_grid = 0, tfw_grid = 0, tbw_grid = 0;
    // refactorization of the tree part in two launches: the wide lower levels
    // with tf_grid CTAs, then the narrow top levels (at most one unit per SM
    // per level) with one CTA per SM, so no unit there shares an SM's FP64
    // pipe; split points in the plain and the fused unit orders
    int tf_split = 0, tf_split_fused = 0, tf_grid_narrow = 0;
    std::vector<int> tree_lvl_units; // factorization units per level of the tree part, lowest level first
    int* ctr_fac = nullptr;          // counter block of the refactorization kernel
    int* ctr_sol = nullptr;          // counter block of the two solve kernels
    int* stall = nullptr;            // failure-injection hook (two ints)
    // Jacobi-sweep preconditioner: row lists of L's off-front entries, work vectors (one instance)
    int* jl_ptr = nullptr;
    int* jl_idx = nullptr;
    void* jac_buf = nullptr;         // 3 n + rel.size() values in factor precision
    // refinement workspace (FP64)
    double* V = nullptr;             // n x (m+1)
    double* Z = nullptr;             // n x m
    double* w = nullptr;
    double* r = nullptr;
    double* red = nullptr;           // reduction scratch + small vectors
    double* h_dev = nullptr;         // small vectors on device
    double* gm = nullptr;            // FGMRES state on the device (kGm* offsets)
    double* pin_flags = nullptr;     // pinned mirror of the convergence flags
    double* kvals = nullptr;         // copy of K made by the last refactor (sliced layout)
    double* stage_vals = nullptr;    // device staging for kkt_step_host
    double* stage_b = nullptr;
    double* stage_x = nullptr;
    double* pin = nullptr;           // pinned host mirror of small results
    double* omega_part = nullptr;    // batched backward error: partial maxima and results
    double* r_batch = nullptr;       // residual vectors of all instances
    double* omega_dev = nullptr;
    double* omega_pin = nullptr;
    DevStat* stat_pin = nullptr;     // pinned host copy of the statistics (sync_stat)
    cudaStream_t work_stream = nullptr;   // own stream for concurrent multi-context batches
    // kkt_step_host: the host buffer for x, copied right after the residual
    // (before the host reads the backward error); x_early_valid: no
    // refinement changed x after that copy
    double* x_early = nullptr;
    int x_early_valid = 0;
    cudaEvent_t done_event = nullptr;
    std::vector<kkt_info> infos;     // per instance
    // launch accounting and optional per-kernel timing
    long long launches = 0;
    int profile = 0;
    std::vector<cudaEvent_t> ev;       // 2 events per recorded launch group
    std::vector<int> ev_kind;
    std::vector<int> ev_count;         // kernels issued by the group
    size_t ev_used = 0;
    // CUDA graphs of the level loops (captured once on a private stream)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t g_factor = nullptr, g_solve = nullptr;
    long long g_factor_kernels = 0, g_solve_kernels = 0;
    cudaGraphExec_t g_ffwd = nullptr, g_bwd = nullptr;     // fused refactor + forward solve; backward solve
    long long g_ffwd_kernels = 0, g_bwd_kernels = 0;
    cudaGraphExec_t g_levels = nullptr;                     // level-launched part only (group refactorization)
    long long g_levels_kernels = 0;
    bool capturing = false;
    // state
    const double* last_vals = nullptr;
    int refactored = 0;
    int refactor_count = 0;
    kkt_info info{};
    int64_t device_bytes = 0;
};

// A group of contexts whose refactorizations run together: the level parts
// on the contexts' own streams, the tree parts in one launch (TreeJob /
// TreeSeg tables and the group's counter block in one device allocation).
struct kkt_group {
    std::vector<kkt_ctx*> ctxs;
    int precision = 0;
    void* dev = nullptr;
    void* jobs = nullptr;
    TreeSeg* segs = nullptr;
    int* gctr = nullptr;
    int nseg = 0, total = 0, grid = 0;
    size_t smem = 0;
    long long spin_limit = 0;
};

namespace {

#define KKT_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return KKT_E_CUDA;           \
    } while (0)

void fill_defaults(kkt_options* o)
{
    std::memset(o, 0, sizeof(*o));
    o->precision = KKT_FP64;
    o->ordering = KKT_ORDER_MINDEG;
    o->user_perm = nullptr;
    o->static_pivot_eps = 0.0;
    o->ruiz_iters = 10;
    o->restart = 30;
    o->max_cycles = 10;
    o->relax_pivots = 16;
    o->relax_zeros = 0.15;
    o->max_pivots = 16;
    o->no_graphs = 0;
    o->tree_min_fronts = 2432;                  // 16 fronts per SM of a 152-SM GB300
    o->spin_limit = 1LL << 23;
    o->precond = KKT_PRECOND_LU;
    o->jacobi_sweeps = 4;
}

kkt_status check_options(const kkt_options& o)
{
    if (o.precision != KKT_FP64 && o.precision != KKT_FP32_IR) return KKT_E_ARG;
    if (o.ordering < 0 || o.ordering > 2) return KKT_E_ARG;
    if (o.ruiz_iters < 0 || o.ruiz_iters > 64) return KKT_E_ARG;
    if (o.restart < 1 || o.restart > kMaxRestart) return KKT_E_ARG;
    if (o.max_cycles < 0) return KKT_E_ARG;
    if (o.max_pivots < 1 || o.max_pivots > 64) return KKT_E_ARG;
    if (o.relax_pivots < 1) return KKT_E_ARG;
    if (o.tree_min_fronts < 0 || o.spin_limit < 1) return KKT_E_ARG;
    if (o.precond != KKT_PRECOND_LU && o.precond != KKT_PRECOND_JACOBI && o.precond != KKT_PRECOND_BLOCK_JACOBI)
        return KKT_E_ARG;
    if (o.jacobi_sweeps < 1 || o.jacobi_sweeps > 1000000) return KKT_E_ARG;
    if (std::isnan(o.static_pivot_eps) || o.static_pivot_eps >= 1.0) return KKT_E_ARG;   // <= 0: the default
    if (!(o.relax_zeros >= 0.0 && o.relax_zeros <= 1.0)) return KKT_E_ARG;
    return KKT_OK;
}

AnalysisOptions to_analysis(const kkt_options& o)
{
    AnalysisOptions a;
    a.ordering = o.ordering;
    a.user_perm = o.user_perm;
    a.relax_small = o.relax_pivots;
    a.relax_zeros = o.relax_zeros;
    a.max_pivots = o.max_pivots;
    return a;
}

size_t elem_size(int precision) { return precision == KKT_FP32_IR ? 4 : 8; }

constexpr size_t kSmemLimit = 220 * 1024;

// Classify fronts per level and lay out the launch lists.
void build_levels(const Analysis& an, size_t es, int nlev, std::vector<LevelGroup>& levels,
                  std::vector<int>& front_ids, std::vector<FrontTile>& tiles, int64_t& scratch_stride,
                  int& max_panel_global, std::vector<int64_t>& inv_off, std::vector<int>& inv,
                  std::vector<int64_t>& f12_off, int64_t& f12_total)
{
    inv_off.assign(an.ns, 0);
    inv.clear();
    f12_off.assign(an.ns, 0);
    f12_total = 0;
    levels.assign(nlev, LevelGroup());
    front_ids.clear();
    tiles.clear();
    scratch_stride = 0;
    max_panel_global = 0;
    for (int l = 0; l < nlev; ++l) {
        LevelGroup& g = levels[l];
        std::vector<int> wl, cl, pl;
        int cmax = 0;
        size_t psmem = 0;
        int allmax = 0, allw = 0;
        for (int t = an.level_ptr[l]; t < an.level_ptr[l + 1]; ++t) {
            int s = an.level_fronts[t];
            int F = an.sn_front[s], w = an.sn_first[s + 1] - an.sn_first[s];
            allmax = std::max(allmax, F);
            allw = std::max(allw, w);
            if (F - w >= kPanelCbMin) {
                pl.push_back(s);
                psmem = std::max(psmem, (size_t)(F * w + w * (F - w)) * es + (size_t)F * sizeof(int));
                g.panel_maxW = std::max(g.panel_maxW, w);
            } else if (F <= kWarpFrontMax) {
                wl.push_back(s);
            } else {
                cl.push_back(s);
                cmax = std::max(cmax, F);
            }
        }
        // a warp per front pays only when the level has enough fronts to fill
        // the GPU; on narrow levels a lone warp cannot hide latency, so small
        // fronts go to the CTA kernels as well
        if ((int)wl.size() < kWarpLevelMin) {
            for (int s : wl) cmax = std::max(cmax, an.sn_front[s]);
            cl.insert(cl.begin(), wl.begin(), wl.end());
            wl.clear();
        }
        std::vector<int> l8, l16, wrest;
        for (int s : wl) {
            const int F = an.sn_front[s];
            const bool leaf = an.child_ptr[s + 1] == an.child_ptr[s];
            (leaf && F <= 8 ? l8 : leaf && F <= 16 ? l16 : wrest).push_back(s);
        }
        for (int s : wl) {
            g.small_maxF = std::max(g.small_maxF, an.sn_front[s]);
            g.small_maxW = std::max(g.small_maxW, an.sn_first[s + 1] - an.sn_first[s]);
        }
        for (int s : wrest) {
            g.wfac_maxF = std::max(g.wfac_maxF, an.sn_front[s]);
            int vol = 0, rs = 0;                  // children's blocks of this front: values, rows
            for (int c = an.child_ptr[s]; c < an.child_ptr[s + 1]; ++c) {
                const int ch = an.child_list[c];
                const int mc = an.sn_front[ch] - (an.sn_first[ch + 1] - an.sn_first[ch]);
                vol += mc * mc;
                rs += mc;
            }
            g.warp_stage_v = std::max(g.warp_stage_v, std::min(vol, kWarpStageV));
            g.warp_stage_r = std::max(g.warp_stage_r, std::min(rs, kWarpStageR));
        }
        for (const std::vector<int>* lst : {&cl, &pl})
            for (int s : *lst) {
                g.big_maxF = std::max(g.big_maxF, an.sn_front[s]);
                g.big_maxW = std::max(g.big_maxW, an.sn_first[s + 1] - an.sn_first[s]);
            }
        g.all_off = (int)front_ids.size();
        for (int t = an.level_ptr[l]; t < an.level_ptr[l + 1]; ++t) front_ids.push_back(an.level_fronts[t]);
        g.all_cnt = (int)(front_ids.size() - g.all_off);
        g.all_maxF = allmax;
        g.all_maxW = allw;
        g.warp_off = (int)front_ids.size();
        front_ids.insert(front_ids.end(), wl.begin(), wl.end());
        g.warp_cnt = (int)wl.size();
        g.leaf8_off = (int)front_ids.size();
        front_ids.insert(front_ids.end(), l8.begin(), l8.end());
        g.leaf8_cnt = (int)l8.size();
        g.leaf16_off = (int)front_ids.size();
        front_ids.insert(front_ids.end(), l16.begin(), l16.end());
        g.leaf16_cnt = (int)l16.size();
        g.wfac_off = (int)front_ids.size();
        front_ids.insert(front_ids.end(), wrest.begin(), wrest.end());
        g.wfac_cnt = (int)wrest.size();
        g.cta_off = (int)front_ids.size();
        front_ids.insert(front_ids.end(), cl.begin(), cl.end());
        g.cta_cnt = (int)cl.size();
        g.cta_maxF = cmax;
        g.panel_off = (int)front_ids.size();
        front_ids.insert(front_ids.end(), pl.begin(), pl.end());
        g.panel_cnt = (int)pl.size();
        g.panel_smem = psmem;
        if (psmem > kSmemLimit) {
            g.panel_global = true;
            scratch_stride = std::max<int64_t>(scratch_stride, (int64_t)(psmem / es));
            max_panel_global = std::max(max_panel_global, g.panel_cnt);
        }
        // gather maps of the panel-class fronts: parent CB row -> child CB row
        for (int s : pl) {
            int F = an.sn_front[s], w = an.sn_first[s + 1] - an.sn_first[s];
            int m = F - w;
            f12_off[s] = f12_total;
            f12_total += (int64_t)w * m;
            inv_off[s] = (int64_t)inv.size();
            for (int c = an.child_ptr[s]; c < an.child_ptr[s + 1]; ++c) {
                int ch = an.child_list[c];
                size_t base = inv.size();
                inv.resize(base + m, -1);
                int mc = an.sn_front[ch] - (an.sn_first[ch + 1] - an.sn_first[ch]);
                for (int t = 0; t < mc; ++t) {
                    int pos = an.rel[an.rel_ptr[ch] + t];
                    if (pos >= w) inv[base + (pos - w)] = t;
                }
            }
        }
        g.tile_off = (int)tiles.size();
        for (int s : pl) {
            int F = an.sn_front[s], w = an.sn_first[s + 1] - an.sn_first[s];
            int m = F - w, nt = (m + kTile - 1) / kTile;
            for (int tj = 0; tj < nt; ++tj)
                for (int ti = 0; ti < nt; ++ti) tiles.push_back(FrontTile{s, ti, tj});
        }
        g.tile_cnt = (int)(tiles.size() - g.tile_off);
    }
    scratch_stride = (scratch_stride + 31) & ~int64_t(31);
}

template <typename T>
DevNum<T>& num_of(kkt_ctx* c);
template <>
DevNum<double>& num_of<double>(kkt_ctx* c) { return c->nd; }
template <>
DevNum<float>& num_of<float>(kkt_ctx* c) { return c->nf; }

enum KernelKind { KK_RUIZ = 0, KK_SCALE, KK_FRONT_WARP, KK_FRONT_CTA, KK_FRONT_PANEL, KK_SCHUR, KK_SOLVE_PRE,
                  KK_SOLVE_FWD, KK_SOLVE_BWD, KK_SOLVE_POST, KK_SPMV, KK_REDUCE, KK_VECTOR, KK_TREE_FACTOR,
                  KK_TREE_FWD, KK_TREE_BWD, KK_JACOBI, KK_FRONT_LEAF, KK_COUNT };
const char* const kKernelNames[KK_COUNT] = {
    "ruiz_kernel", "scale_kernel", "front_warp_kernel", "front_cta_kernel", "front_panel_kernel",
    "schur_tile_kernel", "solve_pre_kernel", "solve_fwd_kernel", "solve_bwd_kernel", "solve_post_kernel",
    "spmv_resid_kernel", "reduction_kernels", "vector_kernels", "tree_factor_kernel", "tree_fwd_kernel",
    "tree_bwd_kernel", "jacobi_kernels", "front_leaf_kernel"};

// Counts kernels and, in profiling mode, brackets the launch group with a
// pair of events on the launching stream.
struct Launch {
    kkt_ctx* c;
    cudaStream_t st;
    int kind, kernels;
    size_t slot = (size_t)-1;
    Launch(kkt_ctx* c_, cudaStream_t st_, int kind_, int kernels_) : c(c_), st(st_), kind(kind_), kernels(kernels_)
    {
        if (!c->capturing) c->launches += kernels;
        if (c->profile && kernels > 0 && !c->capturing) {
            if (c->ev_used + 2 > c->ev.size()) {
                for (int i = 0; i < 512; ++i) {
                    cudaEvent_t e;
                    if (cudaEventCreate(&e) != cudaSuccess) return;
                    c->ev.push_back(e);
                }
                c->ev_kind.resize(c->ev.size() / 2);
                c->ev_count.resize(c->ev.size() / 2);
            }
            slot = c->ev_used / 2;
            c->ev_used += 2;
            c->ev_kind[slot] = kind;
            c->ev_count[slot] = kernels;
            cudaEventRecord(c->ev[2 * slot], st);
        }
    }
    ~Launch()
    {
        if (slot != (size_t)-1) cudaEventRecord(c->ev[2 * slot + 1], st);
    }
};

// Capture a launch sequence into an executable graph on the context's
// private stream (the caller's stream may be the legacy stream, which cannot
// capture). Kernels launched during capture are counted once, per replay.
template <typename F>
kkt_status capture(kkt_ctx* c, cudaGraphExec_t* exec, long long* kernels, F&& body)
{
    if (!c->cap_stream) KKT_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    long long before = c->launches;
    KKT_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    kkt_status s = body(c->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    c->capturing = false;
    if (s != KKT_OK) { if (graph) cudaGraphDestroy(graph); return s; }
    if (e != cudaSuccess) return KKT_E_CUDA;
    size_t nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nodes);
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { *exec = nullptr; return KKT_E_CUDA; }
    *kernels = (long long)nodes;
    c->launches = before;
    return KKT_OK;
}

// fused: the forward substitution of the right-hand side staged in nm.vec
// rides along (warp classes of the level-launched part inside their
// factorization kernels, larger level fronts right after their level, tree
// part inside the persistent kernel)
// with_tree = false: the level-launched part only (a group launches the tree
// parts of all its contexts together); the tree counters are cleared either way.
template <typename T>
kkt_status factor_levels(kkt_ctx* c, DevNum<T>& nm, cudaStream_t st, bool fused = false, bool with_tree = true)
{
    const int* fr = c->fronts_dev;
    const int B = c->batch;
    const int nq = c->tsched.nq;
    if (nq > 0) KKT_CUDA(cudaMemsetAsync(c->ctr_fac, 0, sizeof(int) * (kCtrHead + 2 * (size_t)B * nq), st));
    for (const LevelGroup& g : c->levels) {
        const int fz = fused ? 1 : 0;
        if (g.leaf8_cnt) {
            Launch L(c, st, KK_FRONT_LEAF, 1);
            KKT_CUDA(launch_fronts_leaf<T>(c->sched, nm, fr + g.leaf8_off, g.leaf8_cnt, 8, fz, B, st));
        }
        if (g.leaf16_cnt) {
            Launch L(c, st, KK_FRONT_LEAF, 1);
            KKT_CUDA(launch_fronts_leaf<T>(c->sched, nm, fr + g.leaf16_off, g.leaf16_cnt, 16, fz, B, st));
        }
        if (g.wfac_cnt) {
            Launch L(c, st, KK_FRONT_WARP, 1);
            KKT_CUDA(launch_fronts_warp<T>(c->sched, nm, fr + g.wfac_off, g.wfac_cnt, g.wfac_maxF, g.warp_stage_v,
                                           g.warp_stage_r, fz, B, st));
        }
        if (g.cta_cnt) {
            Launch L(c, st, KK_FRONT_CTA, 1);
            KKT_CUDA(launch_fronts_cta<T>(c->sched, nm, fr + g.cta_off, g.cta_cnt, g.cta_maxF, B, st));
        }
        if (g.panel_cnt) {
            {
                Launch L(c, st, KK_FRONT_PANEL, 1);
                KKT_CUDA(launch_fronts_panel<T>(c->sched, nm, fr + g.panel_off, g.panel_cnt, g.panel_smem,
                                                g.panel_global ? reinterpret_cast<T*>(c->panel_scratch) : nullptr,
                                                c->scratch_stride, B, st));
            }
            Launch L(c, st, KK_SCHUR, 1);
            KKT_CUDA(launch_schur_tiles<T>(c->sched, nm, c->tiles_dev + g.tile_off, g.tile_cnt, g.panel_maxW, B, st));
        }
        // fused: the warp classes did their forward steps; the CTA and panel
        // classes take theirs now, before the next level needs their vectors
        const int nbig = g.cta_cnt + g.panel_cnt;
        if (fused && nbig) {
            Launch L(c, st, KK_SOLVE_FWD, 1);
            KKT_CUDA(launch_solve_fwd_cta<T>(c->sched, nm, fr + g.cta_off, nbig, g.big_maxF, g.big_maxW, B, st));
        }
    }
    if (nq > 0 && with_tree) {
        const int nu = fused ? c->tsched.nunits_fused : c->tsched.nunits;
        const int us = fused ? c->tf_split_fused : c->tf_split;
        if (us > 0) {
            Launch L(c, st, KK_TREE_FACTOR, 1);
            KKT_CUDA(launch_tree_factor<T>(c->sched, c->tsched, nm, B, c->ctr_fac, c->stall, c->opt.spin_limit,
                                           c->tf_grid, c->tf_smem, fused ? 1 : 0, 0, us, 0, st));
        }
        if (us < nu) {
            Launch L(c, st, KK_TREE_FACTOR, 1);
            KKT_CUDA(launch_tree_factor<T>(c->sched, c->tsched, nm, B, c->ctr_fac, c->stall, c->opt.spin_limit,
                                           c->tf_grid_narrow, c->tf_smem, fused ? 1 : 0, us, nu - us, 3, st));
        }
    }
    return KKT_OK;
}

// forward substitution of the level-launched part: fronts with F <= 32 a warp
// each; larger ones (the CTA and panel classes, contiguous in the front
// list) a CTA each
template <typename T>
kkt_status fwd_levels(kkt_ctx* c, const DevNum<T>& nm, int B, cudaStream_t st)
{
    const int* fr = c->fronts_dev;
    for (size_t l = 0; l < c->levels.size(); ++l) {
        const LevelGroup& g = c->levels[l];
        const int nbig = g.cta_cnt + g.panel_cnt;
        if (g.warp_cnt) {
            Launch L(c, st, KK_SOLVE_FWD, 1);
            KKT_CUDA(launch_solve_fwd<T>(c->sched, nm, fr + g.warp_off, g.warp_cnt, g.small_maxF, g.small_maxW, B, st));
        }
        if (nbig) {
            Launch L(c, st, KK_SOLVE_FWD, 1);
            KKT_CUDA(launch_solve_fwd_cta<T>(c->sched, nm, fr + g.cta_off, nbig, g.big_maxF, g.big_maxW, B, st));
        }
    }
    return KKT_OK;
}

// backward substitution (tree part, then the level-launched part); with_fwd:
// the tree part's forward substitution first (the solve path; the fused
// refactorization has done it already)
template <typename T>
kkt_status bwd_levels(kkt_ctx* c, const DevNum<T>& nm, int B, cudaStream_t st, bool with_fwd)
{
    const int* fr = c->fronts_dev;
    const int nq = c->tsched.nq;
    if (nq > 0) {
        KKT_CUDA(cudaMemsetAsync(c->ctr_sol, 0, sizeof(int) * (kCtrHead + 2 * (size_t)B * nq), st));
        if (with_fwd) {
            Launch L(c, st, KK_TREE_FWD, 1);
            KKT_CUDA(launch_tree_fwd<T>(c->sched, c->tsched, nm, B, c->ctr_sol, c->opt.spin_limit, c->tfw_grid,
                                        c->tfw_smem, st));
        }
        Launch L(c, st, KK_TREE_BWD, 1);
        KKT_CUDA(launch_tree_bwd<T>(c->sched, c->tsched, nm, B, c->ctr_sol, c->opt.spin_limit, c->tbw_grid,
                                    c->tbw_smem, st));
    }
    for (size_t l = c->levels.size(); l-- > 0;) {
        const LevelGroup& g = c->levels[l];
        const int nbig = g.cta_cnt + g.panel_cnt;
        // the warp class: small childless fronts several per warp, the rest a warp each
        if (g.leaf8_cnt) {
            Launch L(c, st, KK_SOLVE_BWD, 1);
            KKT_CUDA(launch_solve_bwd_leaf<T>(c->sched, nm, fr + g.leaf8_off, g.leaf8_cnt, 8, B, st));
        }
        if (g.leaf16_cnt) {
            Launch L(c, st, KK_SOLVE_BWD, 1);
            KKT_CUDA(launch_solve_bwd_leaf<T>(c->sched, nm, fr + g.leaf16_off, g.leaf16_cnt, 16, B, st));
        }
        if (g.wfac_cnt) {
            Launch L(c, st, KK_SOLVE_BWD, 1);
            KKT_CUDA(launch_solve_bwd<T>(c->sched, nm, fr + g.wfac_off, g.wfac_cnt, g.small_maxF, g.small_maxW, B, st));
        }
        if (nbig) {
            Launch L(c, st, KK_SOLVE_BWD, 1);
            KKT_CUDA(launch_solve_bwd_cta<T>(c->sched, nm, fr + g.cta_off, nbig, g.big_maxF, g.big_maxW, B, st));
        }
    }
    return KKT_OK;
}

template <typename T>
kkt_status solve_levels(kkt_ctx* c, const DevNum<T>& nm, int B, cudaStream_t st)
{
    kkt_status s = fwd_levels<T>(c, nm, B, st);
    return s != KKT_OK ? s : bwd_levels<T>(c, nm, B, st, true);
}

template <typename T>
kkt_status refactor_t(kkt_ctx* c, const double* d_vals, cudaStream_t st)
{
    DevNum<T>& nm = num_of<T>(c);
    nm.vals = d_vals;
    KKT_CUDA(cudaMemsetAsync(c->stat, 0, sizeof(DevStat) * c->batch, st));
    double* dfin = nullptr;
    {
        Launch L(c, st, KK_RUIZ, c->opt.ruiz_iters > 0 ? c->opt.ruiz_iters : 1);
        KKT_CUDA(launch_ruiz(c->sched, d_vals, c->nnz, nm.kcopy, nm.keys, c->slots, c->d_a, c->d_b, c->opt.ruiz_iters,
                             c->stat, &dfin, c->batch, st));
    }
    c->d_final = dfin;
    nm.d = dfin;
    {
        Launch L(c, st, KK_SCALE, 1);
        KKT_CUDA(launch_scale<T>(c->sched, nm, dfin, c->batch, st));
    }
    if (!c->profile && !c->opt.no_graphs) {
        if (!c->g_factor) {
            kkt_status cs = capture(c, &c->g_factor, &c->g_factor_kernels,
                                    [&](cudaStream_t cst) { return factor_levels<T>(c, nm, cst); });
            if (cs != KKT_OK) return cs;
        }
        c->launches += c->g_factor_kernels;
        KKT_CUDA(cudaGraphLaunch(c->g_factor, st));
        return KKT_OK;
    }
    return factor_levels<T>(c, nm, st);
}

// Equilibration, scatter and the level-launched part of the refactorization,
// without the tree part (a group launches the tree parts of its contexts
// together, kkt_refactor_group).
template <typename T>
kkt_status refactor_levels_t(kkt_ctx* c, const double* d_vals, cudaStream_t st)
{
    DevNum<T>& nm = num_of<T>(c);
    nm.vals = d_vals;
    KKT_CUDA(cudaMemsetAsync(c->stat, 0, sizeof(DevStat) * c->batch, st));
    double* dfin = nullptr;
    {
        Launch L(c, st, KK_RUIZ, c->opt.ruiz_iters > 0 ? c->opt.ruiz_iters : 1);
        KKT_CUDA(launch_ruiz(c->sched, d_vals, c->nnz, nm.kcopy, nm.keys, c->slots, c->d_a, c->d_b, c->opt.ruiz_iters,
                             c->stat, &dfin, c->batch, st));
    }
    c->d_final = dfin;
    nm.d = dfin;
    {
        Launch L(c, st, KK_SCALE, 1);
        KKT_CUDA(launch_scale<T>(c->sched, nm, dfin, c->batch, st));
    }
    if (!c->profile && !c->opt.no_graphs) {
        if (!c->g_levels) {
            kkt_status cs = capture(c, &c->g_levels, &c->g_levels_kernels,
                                    [&](cudaStream_t cst) { return factor_levels<T>(c, nm, cst, false, false); });
            if (cs != KKT_OK) return cs;
        }
        c->launches += c->g_levels_kernels;
        KKT_CUDA(cudaGraphLaunch(c->g_levels, st));
        return KKT_OK;
    }
    return factor_levels<T>(c, nm, st, false, false);
}

// Solve every instance (captured graph of the level loops), or only instance
// `inst` (direct launches; b and x then point at that instance's vectors).
template <typename T>
kkt_status solve_t(kkt_ctx* c, const double* b, double* x, cudaStream_t st, int inst)
{
    const DevNum<T> nm = inst < 0 ? num_of<T>(c) : num_of<T>(c).at(inst);
    const int B = inst < 0 ? c->batch : 1;
    {
        Launch L(c, st, KK_SOLVE_PRE, 1);
        KKT_CUDA(launch_solve_pre<T>(c->sched, nm, b, B, st));
    }
    if (inst < 0 && !c->profile && !c->opt.no_graphs) {
        if (!c->g_solve) {
            kkt_status cs = capture(c, &c->g_solve, &c->g_solve_kernels,
                                    [&](cudaStream_t cst) { return solve_levels<T>(c, nm, B, cst); });
            if (cs != KKT_OK) return cs;
        }
        c->launches += c->g_solve_kernels;
        KKT_CUDA(cudaGraphLaunch(c->g_solve, st));
    } else {
        kkt_status ls = solve_levels<T>(c, nm, B, st);
        if (ls != KKT_OK) return ls;
    }
    {
        Launch L(c, st, KK_SOLVE_POST, 1);
        KKT_CUDA(launch_solve_post<T>(c->sched, nm, x, B, st));
    }
    return KKT_OK;
}

// Refactorization with the forward substitution of b riding along, then the
// backward substitution into x: the first solve of kkt_refactor_refine.
template <typename T>
kkt_status refactor_solve_t(kkt_ctx* c, const double* d_vals, const double* b, double* x, cudaStream_t st)
{
    DevNum<T>& nm = num_of<T>(c);
    nm.vals = d_vals;
    const int B = c->batch;
    KKT_CUDA(cudaMemsetAsync(c->stat, 0, sizeof(DevStat) * B, st));
    double* dfin = nullptr;
    {
        Launch L(c, st, KK_RUIZ, c->opt.ruiz_iters > 0 ? c->opt.ruiz_iters : 1);
        KKT_CUDA(launch_ruiz(c->sched, d_vals, c->nnz, nm.kcopy, nm.keys, c->slots, c->d_a, c->d_b, c->opt.ruiz_iters,
                             c->stat, &dfin, B, st));
    }
    c->d_final = dfin;
    nm.d = dfin;
    {
        Launch L(c, st, KK_SCALE, 1);
        KKT_CUDA(launch_scale<T>(c->sched, nm, dfin, B, st));
    }
    {
        Launch L(c, st, KK_SOLVE_PRE, 1);
        KKT_CUDA(launch_solve_pre<T>(c->sched, nm, b, B, st));
    }
    if (!c->profile && !c->opt.no_graphs) {
        if (!c->g_ffwd) {
            kkt_status cs = capture(c, &c->g_ffwd, &c->g_ffwd_kernels,
                                    [&](cudaStream_t cst) { return factor_levels<T>(c, nm, cst, true); });
            if (cs != KKT_OK) return cs;
        }
        if (!c->g_bwd) {
            kkt_status cs = capture(c, &c->g_bwd, &c->g_bwd_kernels,
                                    [&](cudaStream_t cst) { return bwd_levels<T>(c, nm, B, cst, false); });
            if (cs != KKT_OK) return cs;
        }
        c->launches += c->g_ffwd_kernels + c->g_bwd_kernels;
        KKT_CUDA(cudaGraphLaunch(c->g_ffwd, st));
        KKT_CUDA(cudaGraphLaunch(c->g_bwd, st));
    } else {
        kkt_status s = factor_levels<T>(c, nm, st, true);
        if (s == KKT_OK) s = bwd_levels<T>(c, nm, B, st, false);
        if (s != KKT_OK) return s;
    }
    Launch L(c, st, KK_SOLVE_POST, 1);
    KKT_CUDA(launch_solve_post<T>(c->sched, nm, x, B, st));
    return KKT_OK;
}

kkt_status do_refactor(kkt_ctx* c, const double* d_vals, cudaStream_t st)
{
    c->info.status = KKT_OK;
    kkt_status s = c->opt.precision == KKT_FP32_IR ? refactor_t<float>(c, d_vals, st) : refactor_t<double>(c, d_vals, st);
    if (s == KKT_OK) {
        c->last_vals = c->kvals;
        c->refactored = 1;
        c->refactor_count++;
    }
    return s;
}

kkt_status do_solve(kkt_ctx* c, const double* b, double* x, cudaStream_t st, int inst = -1)
{
    return c->opt.precision == KKT_FP32_IR ? solve_t<float>(c, b, x, st, inst) : solve_t<double>(c, b, x, st, inst);
}

// Jacobi sweeps for instance inst (b, x: that instance's vectors)
template <typename T>
kkt_status jacobi_t(kkt_ctx* c, const double* b, double* x, cudaStream_t st, int inst)
{
    const DevNum<T> nm = num_of<T>(c).at(inst);
    const int n = c->n;
    const int64_t nrel = std::max<int64_t>((int64_t)c->an.rel.size(), 1);
    T* ya = reinterpret_cast<T*>(c->jac_buf);
    T* yb = ya + n;
    T* xa = yb + n;
    T* t = xa + n;
    (void)nrel;
    {
        Launch L(c, st, KK_SOLVE_PRE, 1);
        KKT_CUDA(launch_solve_pre<T>(c->sched, nm, b, 1, st));
    }
    {
        const int k = 2 + 3 * c->opt.jacobi_sweeps;
        Launch L(c, st, KK_JACOBI, k);
        KKT_CUDA(launch_jacobi<T>(c->sched, nm, c->opt.jacobi_sweeps, c->opt.precond == KKT_PRECOND_BLOCK_JACOBI,
                                  c->jl_ptr, c->jl_idx, ya, yb, xa, t, nullptr,
                                  st));
    }
    Launch L(c, st, KK_SOLVE_POST, 1);
    KKT_CUDA(launch_solve_post<T>(c->sched, nm, x, 1, st));
    return KKT_OK;
}

// z = M^{-1} r with the context's preconditioner; inst < 0: every instance
kkt_status do_precond(kkt_ctx* c, const double* b, double* x, cudaStream_t st, int inst = -1)
{
    if (c->opt.precond == KKT_PRECOND_LU) return do_solve(c, b, x, st, inst);
    const int i0 = inst < 0 ? 0 : inst, i1 = inst < 0 ? c->batch : inst + 1;
    for (int i = i0; i < i1; ++i) {
        const int64_t off = inst < 0 ? (int64_t)i * c->n : 0;
        kkt_status s = c->opt.precision == KKT_FP32_IR ? jacobi_t<float>(c, b + off, x + off, st, i)
                                                        : jacobi_t<double>(c, b + off, x + off, st, i);
        if (s != KKT_OK) return s;
    }
    return KKT_OK;
}

// read back the device statistics of the last refactor into c->info
kkt_status sync_stat(kkt_ctx* c, cudaStream_t st)
{
    const DevStat* hs = c->stat_pin;                      // pinned: a plain asynchronous copy
    KKT_CUDA(cudaMemcpyAsync(c->stat_pin, c->stat, sizeof(DevStat) * c->batch, cudaMemcpyDeviceToHost, st));
    KKT_CUDA(cudaStreamSynchronize(st));
    c->infos.resize(c->batch);
    for (int i = 0; i < c->batch; ++i) {
        c->infos[i].n_perturbed = hs[i].n_perturbed;
        c->infos[i].status = hs[i].timeout ? KKT_E_TIMEOUT : hs[i].numeric_bad ? KKT_E_NUMERIC : KKT_OK;
    }
    c->info.n_perturbed = hs[0].n_perturbed;
    if (hs[0].numeric_bad) c->info.status = KKT_E_NUMERIC;
    for (int i = 0; i < c->batch; ++i)
        if (hs[i].timeout) c->info.status = KKT_E_TIMEOUT;
    return KKT_OK;
}

// ||K||_inf of instance inst from the device statistics (synchronizes)
kkt_status knorm_of(kkt_ctx* c, cudaStream_t st, double* knorm, int inst = 0)
{
    unsigned long long bits = 0;
    KKT_CUDA(cudaMemcpyAsync(&bits, &c->stat[inst].knorm_bits, sizeof(bits), cudaMemcpyDeviceToHost, st));
    KKT_CUDA(cudaStreamSynchronize(st));
    std::memcpy(knorm, &bits, sizeof(*knorm));
    return KKT_OK;
}

// ||a||_inf and ||a||_2^2 on the host (synchronizes)
kkt_status norms_host(kkt_ctx* c, const double* a, double* mx, double* sq, cudaStream_t st)
{
    double* out = c->red;
    {
        Launch L(c, st, KK_REDUCE, 2);
        KKT_CUDA(launch_norms(c->n, a, out, st));
    }
    KKT_CUDA(cudaMemcpyAsync(c->pin, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    KKT_CUDA(cudaStreamSynchronize(st));
    *mx = c->pin[0];
    *sq = c->pin[1];
    return KKT_OK;
}

// FGMRES(m) refinement of instance `inst` from the current x (b, x point at
// that instance's vectors). Fills out (iters, backward_err, rel_resid2).
// The Arnoldi process runs on the device (classical Gram-Schmidt twice, the
// Hessenberg column, the Givens rotations and the convergence test in one
// small kernel, the least-squares solve in another): the host issues step
// j + 1 before it reads step j's flag, so the device never waits for the host
// inside a cycle, and one read of the residual norms per cycle decides the
// restart. A step issued after convergence only writes basis columns and
// Hessenberg entries beyond the k used.
kkt_status fgmres_inst(kkt_ctx* c, int inst, const double* b, double* x, double tol, kkt_info* out, cudaStream_t st)
{
    const int n = c->n;
    const int m = c->opt.restart;
    const double* K = c->kvals + (int64_t)inst * c->slots;
    const int pinst = c->batch == 1 ? -1 : inst;     // one instance: the solve replays its captured graph
    kkt_status s;
    double knorm = 0.0;
    if ((s = knorm_of(c, st, &knorm, inst)) != KKT_OK) return s;
    double bmax, bsq, xmax, xsq, rmax, rsq;
    if ((s = norms_host(c, b, &bmax, &bsq, st)) != KKT_OK) return s;
    {
        Launch L(c, st, KK_SPMV, 1);
        KKT_CUDA(launch_spmv_resid(c->sched, K, x, b, c->r, st));
    }
    if ((s = norms_host(c, c->r, &rmax, &rsq, st)) != KKT_OK) return s;
    if ((s = norms_host(c, x, &xmax, &xsq, st)) != KKT_OK) return s;
    auto omega_of = [&](double rm, double xm) {
        double den = knorm * xm + bmax;
        return den > 0 ? rm / den : (den == 0 ? rm : den);           // a NaN norm gives NaN
    };
    double omega = omega_of(rmax, xmax);
    int total = 0;
    double* H = c->gm + kGmH;
    double* cs = c->gm + kGmCs;
    double* sn = c->gm + kGmSn;
    double* g = c->gm + kGmG;
    double* y = c->gm + kGmY;
    double* scale = c->gm + kGmScale;
    double* flag = c->gm + kGmFlag;
    double* nrm = c->red + 4096;
    cudaEvent_t evs[2] = {nullptr, nullptr};
    for (int e = 0; e < 2; ++e)
        if (cudaEventCreateWithFlags(&evs[e], cudaEventDisableTiming) != cudaSuccess) {
            if (evs[0]) cudaEventDestroy(evs[0]);
            return KKT_E_CUDA;
        }
    struct EvGuard { cudaEvent_t* e; ~EvGuard() { cudaEventDestroy(e[0]); cudaEventDestroy(e[1]); } } guard{evs};
    for (int cyc = 0; cyc < c->opt.max_cycles && omega > tol && std::isfinite(omega); ++cyc) {
        double beta = std::sqrt(rsq);
        if (beta == 0.0) break;
        const double target = tol * (knorm * xmax + bmax);
        {
            Launch L(c, st, KK_VECTOR, 2);
            KKT_CUDA(launch_fgmres_start(m, beta, g, scale, st));
            KKT_CUDA(launch_scal_copy(n, c->r, c->V, scale, 1, st));
        }
        int k = m;
        for (int j = 0; j < m; ++j) {
            double* vj = c->V + (int64_t)j * n;
            double* zj = c->Z + (int64_t)j * n;
            if ((s = do_precond(c, vj, zj, st, pinst)) != KKT_OK) return s;
            {
                Launch L(c, st, KK_SPMV, 1);
                KKT_CUDA(launch_spmv(c->sched, K, zj, c->w, st));
            }
            // classical Gram-Schmidt, twice (CGS2): h1 into the Hessenberg column, h2 added by the step kernel
            double* col = H + (int64_t)j * kGmLd;
            {
                Launch L(c, st, KK_REDUCE, 2);
                KKT_CUDA(launch_multidot(n, c->V, n, j + 1, c->w, c->red, st));
            }
            KKT_CUDA(cudaMemcpyAsync(col, c->red, (j + 1) * sizeof(double), cudaMemcpyDeviceToDevice, st));
            {
                Launch L(c, st, KK_VECTOR, 1);
                KKT_CUDA(launch_multiaxpy(n, c->w, c->V, n, j + 1, c->red, st));
            }
            {
                Launch L(c, st, KK_REDUCE, 2);
                KKT_CUDA(launch_multidot(n, c->V, n, j + 1, c->w, c->red, st));
            }
            {
                Launch L(c, st, KK_VECTOR, 1);
                KKT_CUDA(launch_multiaxpy(n, c->w, c->V, n, j + 1, c->red, st));
            }
            {
                Launch L(c, st, KK_REDUCE, 2);
                KKT_CUDA(launch_norms(n, c->w, nrm, st));
            }
            {
                Launch L(c, st, KK_VECTOR, 2);
                KKT_CUDA(launch_fgmres_givens(j, kGmLd, c->red, nrm, H, cs, sn, g, scale, flag, target, st));
                if (j + 1 < m) KKT_CUDA(launch_scal_copy(n, c->w, c->V + (int64_t)(j + 1) * n, scale, 1, st));
            }
            KKT_CUDA(cudaMemcpyAsync(c->pin_flags + j, flag + j, sizeof(double), cudaMemcpyDeviceToHost, st));
            KKT_CUDA(cudaEventRecord(evs[j & 1], st));
            if (j > 0) {                               // step j - 1 has (nearly) finished while j was issued
                KKT_CUDA(cudaEventSynchronize(evs[(j - 1) & 1]));
                if (c->pin_flags[j - 1] != 0.0) { k = j; break; }
            }
        }
        if (k == m) {                                  // no earlier flag: the last step decides nothing more
            KKT_CUDA(cudaEventSynchronize(evs[(m - 1) & 1]));
        }
        total += k;
        {
            Launch L(c, st, KK_VECTOR, 2);
            KKT_CUDA(launch_fgmres_lsq(k, kGmLd, H, g, y, st));
            KKT_CUDA(launch_update(n, x, c->Z, n, k, y, st));
        }
        {
            Launch L(c, st, KK_SPMV, 1);
            KKT_CUDA(launch_spmv_resid(c->sched, K, x, b, c->r, st));
        }
        if ((s = norms_host(c, c->r, &rmax, &rsq, st)) != KKT_OK) return s;
        if ((s = norms_host(c, x, &xmax, &xsq, st)) != KKT_OK) return s;
        omega = omega_of(rmax, xmax);
    }
    out->iters = total;
    out->backward_err = omega;
    out->rel_resid2 = bsq > 0 ? std::sqrt(rsq / bsq) : std::sqrt(rsq);
    if (!std::isfinite(omega)) return KKT_E_NUMERIC;
    if (omega > tol) return KKT_E_NOCONV;
    return KKT_OK;
}

// Solve all instances, evaluate every backward error on the device in one
// pass, and run FGMRES only for the instances above tol.
kkt_status refine_tail(kkt_ctx* c, const double* b, double* x, double tol, kkt_info* info, cudaStream_t st);

kkt_status do_refine(kkt_ctx* c, const double* b, double* x, double tol, kkt_info* info, cudaStream_t st)
{
    kkt_status s;
    if ((s = do_precond(c, b, x, st)) != KKT_OK) return s;
    return refine_tail(c, b, x, tol, info, st);
}

// Refactor and refine in one call: with the exact preconditioner and a tree
// part, the first solve's forward substitution rides along the
// refactorization; then residual, backward error and FGMRES as kkt_refine.
kkt_status do_refactor_refine(kkt_ctx* c, const double* d_vals, const double* b, double* x, double tol,
                              kkt_info* info, cudaStream_t st)
{
    if (c->opt.precond != KKT_PRECOND_LU || c->tsched.nq == 0) {
        kkt_status s = do_refactor(c, d_vals, st);
        return s != KKT_OK ? s : do_refine(c, b, x, tol, info, st);
    }
    c->info.status = KKT_OK;
    kkt_status s = c->opt.precision == KKT_FP32_IR ? refactor_solve_t<float>(c, d_vals, b, x, st)
                                                  : refactor_solve_t<double>(c, d_vals, b, x, st);
    if (s != KKT_OK) return s;
    c->last_vals = c->kvals;
    c->refactored = 1;
    c->refactor_count++;
    return refine_tail(c, b, x, tol, info, st);
}

kkt_status refine_tail(kkt_ctx* c, const double* b, double* x, double tol, kkt_info* info, cudaStream_t st)
{
    kkt_status s;
    {
        Launch L(c, st, KK_SPMV, 2);
        KKT_CUDA(launch_resid_omega(c->sched, c->kvals, c->slots, x, b,
                                    c->r_batch, c->omega_part, c->stat, c->omega_dev, c->batch, st));
    }
    if (c->x_early)
        KKT_CUDA(cudaMemcpyAsync(c->x_early, x, sizeof(double) * c->n * c->batch, cudaMemcpyDeviceToHost, st));
    KKT_CUDA(cudaMemcpyAsync(c->omega_pin, c->omega_dev, sizeof(double) * c->batch, cudaMemcpyDeviceToHost, st));
    if ((s = sync_stat(c, st)) != KKT_OK) return s;      // synchronizes st
    c->x_early_valid = c->x_early != nullptr;
    if (c->info.status == KKT_E_TIMEOUT) {                // a bounded device wait gave up: no valid x
        for (int i = 0; i < c->batch; ++i) {
            c->infos[i].iters = 0;
            c->infos[i].backward_err = c->omega_pin[i];
            c->infos[i].rel_resid2 = -1.0;
        }
        if (info)
            for (int i = 0; i < c->batch; ++i) info[i] = c->infos[i];
        return KKT_E_TIMEOUT;
    }
    kkt_status worst = KKT_OK;
    for (int i = 0; i < c->batch; ++i) {
        kkt_info& inf = c->infos[i];
        inf.iters = 0;
        inf.backward_err = c->omega_pin[i];
        inf.rel_resid2 = -1.0;                            // computed only when refinement runs
        kkt_status si = KKT_OK;
        if (!(c->omega_pin[i] <= tol)) {
            c->x_early_valid = 0;                          // refinement changes x
            const int64_t off = (int64_t)i * c->n;
            si = fgmres_inst(c, i, b + off, x + off, tol, &inf, st);
            if (si != KKT_OK && si != KKT_E_NOCONV && si != KKT_E_NUMERIC) return si;
        }
        if (inf.status == KKT_E_NUMERIC) si = KKT_E_NUMERIC;
        inf.refactor_count = c->refactor_count;
        inf.launches = c->launches;
        if (si == KKT_E_NUMERIC || (si == KKT_E_NOCONV && worst == KKT_OK)) worst = si;
    }
    c->info.iters = c->infos[0].iters;
    c->info.backward_err = c->infos[0].backward_err;
    c->info.rel_resid2 = c->infos[0].rel_resid2;
    if (info)
        for (int i = 0; i < c->batch; ++i) info[i] = c->infos[i];
    return worst;
}

template <typename T>
kkt_status group_tables(kkt_group* g)
{
    std::vector<TreeJob<T>> jobs;
    std::vector<int> job_ctx;
    for (size_t i = 0; i < g->ctxs.size(); ++i) {
        kkt_ctx* c = g->ctxs[i];
        if (c->tsched.nq == 0 || c->tree_lvl_units.empty()) continue;
        TreeJob<T> j;
        j.s = c->sched;
        j.ts = c->tsched;
        j.nm = num_of<T>(c);
        j.B = c->batch;
        j.ctr = c->ctr_fac;
        jobs.push_back(j);
        job_ctx.push_back((int)i);
        g->smem = std::max(g->smem, c->tf_smem);
        g->spin_limit = std::max(g->spin_limit, c->opt.spin_limit);
    }
    // segments: one per (context, tree level), ordered by height below the
    // context's root, the highest first; within a height, context order
    std::vector<TreeSeg> segs;
    std::vector<std::vector<int>> ul0(jobs.size());
    int maxL = 0;
    for (size_t j = 0; j < jobs.size(); ++j) {
        const std::vector<int>& u = g->ctxs[job_ctx[j]]->tree_lvl_units;
        ul0[j].assign(u.size() + 1, 0);
        for (size_t l = 0; l < u.size(); ++l) ul0[j][l + 1] = ul0[j][l] + u[l];
        maxL = std::max(maxL, (int)u.size());
    }
    int64_t total = 0;
    for (int h = maxL - 1; h >= 0; --h)
        for (size_t j = 0; j < jobs.size(); ++j) {
            const std::vector<int>& u = g->ctxs[job_ctx[j]]->tree_lvl_units;
            const int L = (int)u.size();
            if (h >= L) continue;
            const int l = L - 1 - h;
            if (u[l] == 0) continue;
            segs.push_back(TreeSeg{(int)total, (int)j, ul0[j][l]});
            total += (int64_t)u[l] * jobs[j].B;
        }
    if (total > INT32_MAX) return KKT_E_ARG;
    g->nseg = (int)segs.size();
    g->total = (int)total;
    const size_t jb = (sizeof(TreeJob<T>) * std::max<size_t>(jobs.size(), 1) + 255) & ~size_t(255);
    const size_t sb = (sizeof(TreeSeg) * std::max<size_t>(segs.size(), 1) + 255) & ~size_t(255);
    if (cudaMalloc(&g->dev, jb + sb + 256) != cudaSuccess) {
        cudaGetLastError();
        g->dev = nullptr;
        return KKT_E_NOMEM;
    }
    g->jobs = g->dev;
    g->segs = reinterpret_cast<TreeSeg*>(static_cast<char*>(g->dev) + jb);
    g->gctr = reinterpret_cast<int*>(static_cast<char*>(g->dev) + jb + sb);
    cudaStream_t ust = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&ust, cudaStreamNonBlocking);
    if (e == cudaSuccess && !jobs.empty())
        e = cudaMemcpyAsync(g->jobs, jobs.data(), sizeof(TreeJob<T>) * jobs.size(), cudaMemcpyHostToDevice, ust);
    if (e == cudaSuccess && !segs.empty())
        e = cudaMemcpyAsync(g->segs, segs.data(), sizeof(TreeSeg) * segs.size(), cudaMemcpyHostToDevice, ust);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->gctr, 0, 256, ust);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ust);
    if (ust) cudaStreamDestroy(ust);
    if (e == cudaSuccess && g->total > 0) e = tree_grid<T>(3, g->smem, &g->grid);
    return e == cudaSuccess ? KKT_OK : KKT_E_CUDA;
}

// the pivot reciprocal of the factorization and backward kernels, elementwise
template <typename T>
__global__ void pivot_rcp_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = pivot_rcp(in[i]);
}

}  // namespace

// ======================================================================== C ABI

extern "C" {

void kkt_default_options(kkt_options* opt)
{
    if (opt) fill_defaults(opt);
}

const char* kkt_status_string(kkt_status s)
{
    switch (s) {
    case KKT_OK: return "ok";
    case KKT_E_ARG: return "invalid argument";
    case KKT_E_CUDA: return "CUDA error";
    case KKT_E_NOMEM: return "out of memory";
    case KKT_E_STATE: return "call out of order";
    case KKT_E_STRUCT: return "invalid sparsity pattern";
    case KKT_E_NOCONV: return "refinement did not converge";
    case KKT_E_TIMEOUT: return "device wait timed out";
    case KKT_E_NUMERIC: return "NaN or Inf encountered";
    }
    return "unknown status";
}

static int64_t plan_bytes(const Analysis& an, int n, int64_t nnz, const kkt_options& o, int64_t tiles, int64_t fronts,
                          int64_t scratch, int64_t ninv, int64_t nf12, const TreePlan& tp, const SellPlan& sp,
                          int64_t B = 1)
{
    const int64_t es = (int64_t)elem_size(o.precision);
    int64_t b = 0;
    auto add = [&](int64_t x) { b += (x + 255) & ~int64_t(255); };
    add((n + 1) * 4); add(nnz * 4); add(n * 4);
    add((an.ns + 1) * 4); add(an.ns * 4); add((an.ns + 1) * 8); add((int64_t)an.rows.size() * 4);
    add((an.ns + 1) * 4); add((int64_t)an.child_list.size() * 4);
    add((an.ns + 1) * 8); add(nnz * 4); add(nnz * 4);
    add((an.ns + 1) * 8); add((int64_t)an.rel.size() * 4);
    add((an.ns + 1) * 8); add((an.ns + 1) * 8);
    add(fronts * 4); add(tiles * (int64_t)sizeof(FrontTile));
    add(B * (int64_t)sizeof(DevStat));
    add(B * n * 8); add(B * n * 8);
    add(B * sp.slots * es); add(B * an.panel_total * es); add(B * std::max<int64_t>(an.cb_total, 1) * es);
    add(B * n * es); add(B * std::max<int64_t>((int64_t)an.rel.size(), 1) * es);
    add(B * scratch * es);
    add((int64_t)n * (o.restart + 1) * 8); add((int64_t)n * o.restart * 8); add(n * 8); add(n * 8);
    add((int64_t)(kRedScratch + 4096 + 8) * 8);
    add((int64_t)(8 + 2 * (kMaxRestart + 2)) * 8);
    add((int64_t)kGmSize * 8);
    add(B * sp.slots * 8); add(B * nnz * 8); add(B * n * 8); add(B * n * 8);
    add(an.ns * 4); add(an.ns * 8); add(std::max<int64_t>(ninv, 1) * 4);
    add(an.ns * 8); add(B * std::max<int64_t>(nf12, 1) * es);
    add(B * n * 8); add(B * (int64_t)resid_blocks(n) * 4 * 8); add(B * 8);
    const int64_t nq = (int64_t)tp.fr.size();
    add(nq * (int64_t)sizeof(TreeFront)); add((int64_t)tp.kid.size() * (int64_t)sizeof(TreeKid));
    add((int64_t)tp.unit.size() * (int64_t)sizeof(TreeUnit)); add((int64_t)tp.inv.size() * 4);
    add((int64_t)tp.unit_fused.size() * (int64_t)sizeof(TreeUnit));
    add((int64_t)tp.bwd_chain.size() * 4); add((int64_t)tp.bwd_chain_ptr.size() * 4);
    add((kCtrHead + 2 * B * nq) * 4); add((kCtrHead + 2 * B * nq) * 4); add(2 * 4);
    add((n + 1) * 4); add(std::max<int64_t>((int64_t)an.rel.size(), 1) * 4);
    add((3 * (int64_t)n + std::max<int64_t>((int64_t)an.rel.size(), 1)) * es);
    add(((int64_t)sp.nslices + 1) * 8); add((int64_t)sp.nslices * 32 * 4); add(sp.slots * 4); add(sp.slots * 4);
    add(B * sp.slots * 2);
    return b;
}

kkt_status kkt_plan(int32_t n, const int32_t* h_rowptr, const int32_t* h_colidx, const kkt_options* opt,
                    kkt_plan_info* out)
{
    if (n <= 0 || !h_rowptr || !h_colidx || !out) return KKT_E_ARG;
    kkt_options o;
    if (opt) o = *opt; else fill_defaults(&o);
    if (check_options(o) != KKT_OK) return KKT_E_ARG;
    try {
        Analysis an;
        std::string err = analyze_pattern(n, h_rowptr, h_colidx, to_analysis(o), an);
        if (!err.empty()) return (err.find("user") != std::string::npos) ? KKT_E_ARG : KKT_E_STRUCT;
        std::vector<LevelGroup> lv;
        std::vector<int> fids;
        std::vector<FrontTile> tiles;
        int64_t stride = 0;
        int mpg = 0;
        std::vector<int64_t> inv_off, f12_off;
        std::vector<int> inv;
        int64_t f12_total = 0;
        TreePlan tp;
        build_tree(an, o.tree_min_fronts, elem_size(o.precision), tp);
        build_levels(an, elem_size(o.precision), tp.split, lv, fids, tiles, stride, mpg, inv_off, inv, f12_off,
                     f12_total);
        SellPlan sp;
        build_sell(n, h_rowptr, h_colidx, kSellWindow, sp);
        std::memset(out, 0, sizeof(*out));
        out->n = n;
        out->nnz = an.nnz;
        out->nnz_lu = an.nnz_l + an.nnz_u;
        out->stored_factor = an.stored_factor;
        out->n_fronts = an.ns;
        out->n_levels = an.n_levels;
        out->max_front = an.max_front;
        out->max_pivots = an.max_pivots;
        out->flops = an.flops;
        out->flops_exact = an.flops_exact;
        out->device_bytes = plan_bytes(an, n, an.nnz, o, (int64_t)tiles.size(), (int64_t)fids.size(),
                                       stride * mpg, (int64_t)inv.size(), f12_total, tp, sp);
        out->tree_levels = an.n_levels - tp.split;
        out->tree_units = (int)tp.unit.size();
        out->tree_bytes = tp.alg_bytes;
        out->tree_nnz_k = tp.nnz_k;
        out->tree_nnz_lu = tp.nnz_lu;
        out->tree_pivots = tp.pivots;
    } catch (const std::bad_alloc&) {
        return KKT_E_NOMEM;
    } catch (...) {
        return KKT_E_ARG;
    }
    return KKT_OK;
}

kkt_status kkt_plan_fronts(int32_t n, const int32_t* h_rowptr, const int32_t* h_colidx, const kkt_options* opt,
                           int32_t capacity, int32_t* h_order, int32_t* h_pivots, int32_t* count)
{
    if (n <= 0 || !h_rowptr || !h_colidx || !count || capacity < 0) return KKT_E_ARG;
    if (capacity > 0 && (!h_order || !h_pivots)) return KKT_E_ARG;
    kkt_options o;
    if (opt) o = *opt; else fill_defaults(&o);
    if (check_options(o) != KKT_OK) return KKT_E_ARG;
    try {
        Analysis an;
        std::string err = analyze_pattern(n, h_rowptr, h_colidx, to_analysis(o), an);
        if (!err.empty()) return (err.find("user") != std::string::npos) ? KKT_E_ARG : KKT_E_STRUCT;
        *count = an.ns;
        for (int s = 0; s < an.ns && s < capacity; ++s) {
            h_order[s] = an.sn_front[s];
            h_pivots[s] = an.sn_first[s + 1] - an.sn_first[s];
        }
    } catch (const std::bad_alloc&) {
        return KKT_E_NOMEM;
    } catch (...) {
        return KKT_E_ARG;
    }
    return KKT_OK;
}

static kkt_status analyze_impl(int32_t n, int32_t n_primal, const int32_t* h_rowptr, const int32_t* h_colidx,
                               const kkt_options* opt, int32_t batch, kkt_ctx** out)
{
    if (!out || n <= 0 || !h_rowptr || !h_colidx || n_primal < 0 || n_primal > n || batch < 1) return KKT_E_ARG;
    *out = nullptr;
    kkt_ctx* c = nullptr;
    try {
        c = new kkt_ctx();
    } catch (...) {
        return KKT_E_NOMEM;
    }
    if (opt) c->opt = *opt; else fill_defaults(&c->opt);
    if (check_options(c->opt) != KKT_OK) { delete c; return KKT_E_ARG; }
    c->opt.user_perm = nullptr;
    c->n = n;
    c->n_primal = n_primal;
    c->batch = batch;
    const int64_t B = batch;
    std::vector<int> fids;
    std::vector<FrontTile> tiles;
    std::vector<int64_t> inv_off, f12_off;
    std::vector<int> inv;
    int64_t f12_total = 0;
    TreePlan tp;
    SellPlan sp;
    std::vector<int> asm_src_sell;
    try {
        std::string err = analyze_pattern(n, h_rowptr, h_colidx, to_analysis(opt ? *opt : c->opt), c->an);
        if (!err.empty()) {
            kkt_status s = (err.find("user") != std::string::npos) ? KKT_E_ARG : KKT_E_STRUCT;
            delete c;
            return s;
        }
        // a level of a batched context carries `batch` times the fronts of one
        // instance: it stays level-launched once fronts x batch reach the threshold
        const int per_instance = (c->opt.tree_min_fronts + batch - 1) / batch;
        build_tree(c->an, per_instance, elem_size(c->opt.precision), tp);
        build_levels(c->an, elem_size(c->opt.precision), tp.split, c->levels, fids, tiles, c->scratch_stride,
                     c->max_panel_global, inv_off, inv, f12_off, f12_total);
        // K's per-refactor copies live in the sliced layout: the assembly reads them at slots
        build_sell(n, h_rowptr, h_colidx, kSellWindow, sp);
        asm_src_sell.resize(c->an.asm_src.size());
        for (size_t e = 0; e < asm_src_sell.size(); ++e) asm_src_sell[e] = sp.csr2sell[c->an.asm_src[e]];
    } catch (...) {
        delete c;
        return KKT_E_NOMEM;
    }
    static std::once_flag once;
    static cudaError_t cfg_err = cudaSuccess;
    std::call_once(once, [] { cfg_err = configure_kernels(); });
    if (cfg_err != cudaSuccess) { delete c; return KKT_E_CUDA; }

    const Analysis& an = c->an;
    c->nnz = an.nnz;
    c->slots = sp.slots;
    const int64_t nnz = an.nnz;
    const int64_t slots = sp.slots;
    const int64_t scratch = c->scratch_stride * c->max_panel_global;
    int64_t bytes = plan_bytes(an, n, nnz, c->opt, (int64_t)tiles.size(), (int64_t)fids.size(), scratch,
                               (int64_t)inv.size(), f12_total, tp, sp, B);
    c->device_bytes = bytes;
    if (cudaMalloc(&c->pool.base, (size_t)bytes) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return KKT_E_NOMEM;
    }
    c->pool.size = (size_t)bytes;
    Pool& P = c->pool;
    int* rowptr = P.take<int>(n + 1);
    int* colidx = P.take<int>(nnz);
    int* perm = P.take<int>(n);
    int* sn_first = P.take<int>(an.ns + 1);
    int* sn_front = P.take<int>(an.ns);
    int64_t* rows_ptr = P.take<int64_t>(an.ns + 1);
    int* rows = P.take<int>(an.rows.size());
    int* child_ptr = P.take<int>(an.ns + 1);
    int* child_list = P.take<int>(an.child_list.size());
    int64_t* asm_ptr = P.take<int64_t>(an.ns + 1);
    int* asm_pos = P.take<int>(nnz);
    int* asm_src = P.take<int>(nnz);
    int64_t* rel_ptr = P.take<int64_t>(an.ns + 1);
    int* rel = P.take<int>(an.rel.size());
    int64_t* panel_off = P.take<int64_t>(an.ns + 1);
    int64_t* cb_off = P.take<int64_t>(an.ns + 1);
    c->fronts_dev = P.take<int>(fids.size());
    c->tiles_dev = P.take<FrontTile>(tiles.size());
    c->stat = P.take<DevStat>(B);
    c->d_a = P.take<double>(B * n);
    c->d_b = P.take<double>(B * n);
    const size_t es = elem_size(c->opt.precision);
    const int64_t cb_unit = std::max<int64_t>(an.cb_total, 1);
    const int64_t cbv_unit = std::max<int64_t>((int64_t)an.rel.size(), 1);
    const int64_t f12_unit = std::max<int64_t>(f12_total, 1);
    char* sv = P.take<char>(B * slots * es);
    char* panel = P.take<char>(B * an.panel_total * es);
    char* cb = P.take<char>(B * cb_unit * es);
    char* vec = P.take<char>(B * n * es);
    char* cbv = P.take<char>(B * cbv_unit * es);
    c->panel_scratch = P.take<char>(B * scratch * es);
    c->V = P.take<double>((int64_t)n * (c->opt.restart + 1));
    c->Z = P.take<double>((int64_t)n * c->opt.restart);
    c->w = P.take<double>(n);
    c->r = P.take<double>(n);
    c->red = P.take<double>(kRedScratch + 4096 + 8);
    c->h_dev = P.take<double>(8 + 2 * (kMaxRestart + 2));
    c->gm = P.take<double>(kGmSize);
    c->kvals = P.take<double>(B * slots);
    c->stage_vals = P.take<double>(B * nnz);
    c->stage_b = P.take<double>(B * n);
    c->stage_x = P.take<double>(B * n);
    int* cb_split = P.take<int>(an.ns);
    int64_t* inv_off_d = P.take<int64_t>(an.ns);
    int* inv_d = P.take<int>(std::max<size_t>(inv.size(), 1));
    int64_t* f12_off_d = P.take<int64_t>(an.ns);
    char* f12 = P.take<char>(B * f12_unit * es);
    c->r_batch = P.take<double>(B * n);
    c->omega_part = P.take<double>(B * (int64_t)resid_blocks(n) * 4);
    c->omega_dev = P.take<double>(B);
    const int64_t nq = (int64_t)tp.fr.size();
    TreeFront* tfr = P.take<TreeFront>(nq);
    TreeKid* tkid = P.take<TreeKid>(tp.kid.size());
    TreeUnit* tunit = P.take<TreeUnit>(tp.unit.size());
    TreeUnit* tunit_fused = P.take<TreeUnit>(tp.unit_fused.size());
    int* tinv = P.take<int>(tp.inv.size());
    int* tchain = P.take<int>(tp.bwd_chain.size());
    int* tchain_ptr = P.take<int>(tp.bwd_chain_ptr.size());
    c->ctr_fac = P.take<int>(kCtrHead + 2 * B * nq);
    c->ctr_sol = P.take<int>(kCtrHead + 2 * B * nq);
    c->stall = P.take<int>(2);
    c->jl_ptr = P.take<int>(n + 1);
    c->jl_idx = P.take<int>(std::max<size_t>(an.rel.size(), 1));
    c->jac_buf = P.take<char>((3 * (size_t)n + std::max<size_t>(an.rel.size(), 1)) * es);
    int64_t* sell_off = P.take<int64_t>(sp.nslices + 1);
    int* sell_row = P.take<int>((int64_t)sp.nslices * 32);
    int* sell_ci = P.take<int>(slots);
    int* sell_src = P.take<int>(slots);
    unsigned short* keys = P.take<unsigned short>(B * slots);
    if (P.used > P.size) { kkt_destroy(c); return KKT_E_NOMEM; }
    if (cudaMallocHost(&c->stat_pin, sizeof(DevStat) * B) != cudaSuccess) {
        cudaGetLastError();
        c->stat_pin = nullptr;
        kkt_destroy(c);
        return KKT_E_NOMEM;
    }
    if (cudaMallocHost(&c->pin, sizeof(double) * (4 * (kMaxRestart + 2) + 16 + B + kMaxRestart + 8)) != cudaSuccess) {
        cudaGetLastError();
        c->pin = nullptr;
        kkt_destroy(c);
        return KKT_E_NOMEM;
    }
    // Uploads and clears go through the context's own non-blocking stream and
    // are waited for before kkt_analyze returns: a plain cudaMemcpy from
    // pageable memory (or a cudaMemset) may return before the device holds the
    // data, and is not ordered before work the caller then issues on a
    // non-blocking stream of its own.
    cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        c->cap_stream = nullptr;
        kkt_destroy(c);
        return KKT_E_CUDA;
    }
    cudaStream_t ust = c->cap_stream;
    auto up = [&](void* dst, const void* src, size_t bytes_) {
        return bytes_ ? cudaMemcpyAsync(dst, src, bytes_, cudaMemcpyHostToDevice, ust) : cudaSuccess;
    };
    e = e ? e : up(rowptr, h_rowptr, (n + 1) * 4);
    e = e ? e : up(colidx, h_colidx, nnz * 4);
    e = e ? e : up(perm, an.perm.data(), n * 4);
    e = e ? e : up(sn_first, an.sn_first.data(), (an.ns + 1) * 4);
    e = e ? e : up(sn_front, an.sn_front.data(), an.ns * 4);
    e = e ? e : up(rows_ptr, an.rows_ptr.data(), (an.ns + 1) * 8);
    e = e ? e : up(rows, an.rows.data(), an.rows.size() * 4);
    e = e ? e : up(child_ptr, an.child_ptr.data(), (an.ns + 1) * 4);
    e = e ? e : up(child_list, an.child_list.data(), an.child_list.size() * 4);
    e = e ? e : up(asm_ptr, an.asm_ptr.data(), (an.ns + 1) * 8);
    e = e ? e : up(asm_pos, an.asm_pos.data(), nnz * 4);
    e = e ? e : up(asm_src, asm_src_sell.data(), nnz * 4);
    e = e ? e : up(sell_off, sp.off.data(), (sp.nslices + 1) * 8);
    e = e ? e : up(sell_row, sp.row.data(), (size_t)sp.nslices * 32 * 4);
    e = e ? e : up(sell_ci, sp.ci.data(), slots * 4);
    e = e ? e : up(sell_src, sp.src.data(), slots * 4);
    e = e ? e : up(rel_ptr, an.rel_ptr.data(), (an.ns + 1) * 8);
    e = e ? e : up(rel, an.rel.data(), an.rel.size() * 4);
    e = e ? e : up(panel_off, an.panel_off.data(), (an.ns + 1) * 8);
    e = e ? e : up(cb_off, an.cb_off.data(), (an.ns + 1) * 8);
    e = e ? e : up(c->fronts_dev, fids.data(), fids.size() * 4);
    e = e ? e : up(c->tiles_dev, tiles.data(), tiles.size() * sizeof(FrontTile));
    e = e ? e : up(cb_split, an.cb_split.data(), an.ns * 4);
    e = e ? e : up(inv_off_d, inv_off.data(), an.ns * 8);
    e = e ? e : up(inv_d, inv.data(), inv.size() * 4);
    e = e ? e : up(f12_off_d, f12_off.data(), an.ns * 8);
    e = e ? e : up(tfr, tp.fr.data(), nq * sizeof(TreeFront));
    e = e ? e : up(tkid, tp.kid.data(), tp.kid.size() * sizeof(TreeKid));
    // units with their fronts' descriptors
    std::vector<TreeUnit> h_unit(tp.unit.size()), h_unit_fused(tp.unit_fused.size());
    for (size_t i = 0; i < tp.unit.size(); ++i) h_unit[i] = TreeUnit{tp.fr[tp.unit[i].front], tp.unit[i], 0};
    for (size_t i = 0; i < tp.unit_fused.size(); ++i)
        h_unit_fused[i] = TreeUnit{tp.fr[tp.unit_fused[i].front], tp.unit_fused[i], 0};
    e = e ? e : up(tunit, h_unit.data(), h_unit.size() * sizeof(TreeUnit));
    e = e ? e : up(tunit_fused, h_unit_fused.data(), h_unit_fused.size() * sizeof(TreeUnit));
    e = e ? e : up(tinv, tp.inv.data(), tp.inv.size() * 4);
    e = e ? e : up(tchain, tp.bwd_chain.data(), tp.bwd_chain.size() * 4);
    e = e ? e : up(tchain_ptr, tp.bwd_chain_ptr.data(), tp.bwd_chain_ptr.size() * 4);
    e = e ? e : cudaMemsetAsync(c->stall, 0, 2 * sizeof(int), ust);
    {
        // per step row i: contribution-vector offsets rel_ptr[f] + t of every front f whose
        // contribution row t is i, in increasing order (the gather order of the Jacobi sweeps)
        std::vector<int> jp(n + 1, 0), ji(an.rel.size());
        for (int f = 0; f < an.ns; ++f) {
            const int w = an.sn_first[f + 1] - an.sn_first[f], F = an.sn_front[f];
            for (int t = w; t < F; ++t) jp[an.rows[an.rows_ptr[f] + t] + 1]++;
        }
        for (int i = 0; i < n; ++i) jp[i + 1] += jp[i];
        std::vector<int> fill(jp.begin(), jp.end() - 1);
        for (int f = 0; f < an.ns; ++f) {
            const int w = an.sn_first[f + 1] - an.sn_first[f], F = an.sn_front[f];
            for (int t = w; t < F; ++t) ji[fill[an.rows[an.rows_ptr[f] + t]]++] = (int)(an.rel_ptr[f] + (t - w));
        }
        e = e ? e : up(c->jl_ptr, jp.data(), (n + 1) * 4);
        e = e ? e : up(c->jl_idx, ji.data(), ji.size() * 4);
    }
    e = e ? e : cudaMemsetAsync(c->stat, 0, sizeof(DevStat) * B, ust);
    e = e ? e : cudaStreamSynchronize(ust);
    c->omega_pin = c->pin + 4 * (kMaxRestart + 2) + 16;
    c->pin_flags = c->omega_pin + B;
    c->infos.assign(B, kkt_info{});
    if (e != cudaSuccess) { kkt_destroy(c); return KKT_E_CUDA; }
    DevSched& s = c->sched;
    s.n = n; s.nnz = nnz; s.ns = an.ns;
    s.rowptr = rowptr; s.colidx = colidx; s.perm = perm;
    s.sn_first = sn_first; s.sn_front = sn_front; s.rows_ptr = rows_ptr; s.rows = rows;
    s.child_ptr = child_ptr; s.child_list = child_list;
    s.asm_ptr = asm_ptr; s.asm_pos = asm_pos; s.asm_src = asm_src;
    s.rel_ptr = rel_ptr; s.rel = rel; s.panel_off = panel_off; s.cb_off = cb_off;
    s.cb_split = cb_split; s.inv_off = inv_off_d; s.inv = inv_d; s.f12_off = f12_off_d;
    s.nslices = sp.nslices; s.slots = slots;
    s.sell_off = sell_off; s.sell_row = sell_row; s.sell_ci = sell_ci; s.sell_src = sell_src;
    c->tsched = tp.ts;
    c->tsched.fr = tfr; c->tsched.kid = tkid; c->tsched.unit = tunit; c->tsched.inv = tinv;
    c->tsched.unit_fused = tunit_fused;
    c->tsched.bwd_chain = tchain;
    c->tsched.bwd_chain_ptr = tchain_ptr;
    c->tree_split = tp.split;
    c->tree_bytes = tp.alg_bytes;
    c->tree_nnz_k = tp.nnz_k;
    c->tree_nnz_lu = tp.nnz_lu;
    c->tree_pivots = tp.pivots;
    c->tf_smem = tp.fac_smem; c->tfw_smem = tp.fwd_smem; c->tbw_smem = tp.bwd_smem;
    if (nq > 0) {
        const bool f32 = c->opt.precision == KKT_FP32_IR;
        e = f32 ? tree_grid<float>(0, c->tf_smem, &c->tf_grid) : tree_grid<double>(0, c->tf_smem, &c->tf_grid);
        e = e ? e : f32 ? tree_grid<float>(1, c->tfw_smem, &c->tfw_grid) : tree_grid<double>(1, c->tfw_smem, &c->tfw_grid);
        e = e ? e : f32 ? tree_grid<float>(2, c->tbw_smem, &c->tbw_grid) : tree_grid<double>(2, c->tbw_smem, &c->tbw_grid);
        int dev = 0, nsm = 0;
        e = e ? e : cudaGetDevice(&dev);
        e = e ? e : cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) { kkt_destroy(c); return KKT_E_CUDA; }
        // narrow top: the lowest level from which every level has at most one
        // unit (times the batch) per SM; tree index is level-major from tp.split
        c->tf_grid_narrow = nsm;
        std::vector<int> lev(nq), per_level(an.n_levels, 0);
        for (int l = tp.split, q = 0; l < an.n_levels; ++l)
            for (int t = an.level_ptr[l]; t < an.level_ptr[l + 1]; ++t) lev[q++] = l;
        for (const FrontTile& u : tp.unit) per_level[lev[u.front]]++;
        c->tree_lvl_units.assign(per_level.begin() + tp.split, per_level.end());
        int narrow = an.n_levels;
        for (int l = an.n_levels - 1; l >= tp.split && (int64_t)per_level[l] * B <= nsm; --l) narrow = l;
        auto first_at = [&](const std::vector<FrontTile>& order) {   // both orders ascend by level
            int i = 0;
            while (i < (int)order.size() && lev[order[i].front] < narrow) ++i;
            return i;
        };
        c->tf_split = first_at(tp.unit);
        c->tf_split_fused = first_at(tp.unit_fused);
    }
    double eps = c->opt.static_pivot_eps > 0 ? c->opt.static_pivot_eps
                                             : (c->opt.precision == KKT_FP32_IR ? 1e-7 : 1e-14);
    c->opt.static_pivot_eps = eps;
    if (c->opt.precision == KKT_FP32_IR) {
        DevNum<float>& nm = c->nf;
        nm.sv = reinterpret_cast<float*>(sv); nm.panel = reinterpret_cast<float*>(panel);
        nm.cb = reinterpret_cast<float*>(cb); nm.vec = reinterpret_cast<float*>(vec);
        nm.cbv = reinterpret_cast<float*>(cbv); nm.stat = c->stat; nm.pivot_eps = eps; nm.d = c->d_a;
        nm.kcopy = c->kvals;
        nm.keys = keys;
        nm.f12 = reinterpret_cast<float*>(f12);
        nm.dtmp = c->d_b;
        nm.bs_nnz = nnz; nm.bs_slot = slots; nm.bs_n = n; nm.bs_panel = an.panel_total; nm.bs_cb = cb_unit;
        nm.bs_cbv = cbv_unit; nm.bs_f12 = f12_unit;
    } else {
        DevNum<double>& nm = c->nd;
        nm.sv = reinterpret_cast<double*>(sv); nm.panel = reinterpret_cast<double*>(panel);
        nm.cb = reinterpret_cast<double*>(cb); nm.vec = reinterpret_cast<double*>(vec);
        nm.cbv = reinterpret_cast<double*>(cbv); nm.stat = c->stat; nm.pivot_eps = eps; nm.d = c->d_a;
        nm.kcopy = c->kvals;
        nm.keys = keys;
        nm.f12 = reinterpret_cast<double*>(f12);
        nm.dtmp = c->d_b;
        nm.bs_nnz = nnz; nm.bs_slot = slots; nm.bs_n = n; nm.bs_panel = an.panel_total; nm.bs_cb = cb_unit;
        nm.bs_cbv = cbv_unit; nm.bs_f12 = f12_unit;
    }
    c->info.status = KKT_OK;
    *out = c;
    return KKT_OK;
}

kkt_status kkt_analyze(int32_t n, int32_t n_primal, const int32_t* h_rowptr, const int32_t* h_colidx,
                       const double* h_vals, const kkt_options* opt, kkt_ctx** out)
{
    (void)h_vals;
    return analyze_impl(n, n_primal, h_rowptr, h_colidx, opt, 1, out);
}

kkt_status kkt_analyze_batch(int32_t n, int32_t n_primal, const int32_t* h_rowptr, const int32_t* h_colidx,
                             const kkt_options* opt, int32_t count, kkt_ctx** out)
{
    if (count < 1) return KKT_E_ARG;
    return analyze_impl(n, n_primal, h_rowptr, h_colidx, opt, count, out);
}

kkt_status kkt_refactor(kkt_ctx* c, const double* d_vals, void* stream)
{
    if (!c || !d_vals) return KKT_E_ARG;
    c->info.status = KKT_OK;
    return do_refactor(c, d_vals, (cudaStream_t)stream);
}

kkt_status kkt_solve(kkt_ctx* c, const double* d_rhs, double* d_x, void* stream)
{
    if (!c || !d_rhs || !d_x || d_rhs == d_x) return KKT_E_ARG;
    if (!c->refactored) return KKT_E_STATE;
    return do_solve(c, d_rhs, d_x, (cudaStream_t)stream);
}

kkt_status kkt_refine(kkt_ctx* c, const double* d_rhs, double* d_x, double tol, kkt_info* info, void* stream)
{
    if (!c || !d_rhs || !d_x || d_rhs == d_x || !(tol >= 0)) return KKT_E_ARG;
    if (!c->refactored) return KKT_E_STATE;
    return do_refine(c, d_rhs, d_x, tol, info, (cudaStream_t)stream);
}

kkt_status kkt_refactor_refine(kkt_ctx* c, const double* d_vals, const double* d_rhs, double* d_x, double tol,
                               kkt_info* info, void* stream)
{
    if (!c || !d_vals || !d_rhs || !d_x || d_rhs == d_x || !(tol >= 0)) return KKT_E_ARG;
    return do_refactor_refine(c, d_vals, d_rhs, d_x, tol, info, (cudaStream_t)stream);
}

kkt_status kkt_precondition(kkt_ctx* c, const double* d_rhs, double* d_z, void* stream)
{
    if (!c || !d_rhs || !d_z || d_rhs == d_z) return KKT_E_ARG;
    if (!c->refactored) return KKT_E_STATE;
    return do_precond(c, d_rhs, d_z, (cudaStream_t)stream);
}

kkt_status kkt_solve_checked(kkt_ctx* c, const double* d_rhs, double* d_x, double* h_omega, void* stream)
{
    if (!c || !d_rhs || !d_x || !h_omega || d_rhs == d_x) return KKT_E_ARG;
    if (!c->refactored) return KKT_E_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    kkt_status s = do_solve(c, d_rhs, d_x, st);
    if (s != KKT_OK) return s;
    {
        Launch L(c, st, KK_SPMV, 2);
        KKT_CUDA(launch_resid_omega(c->sched, c->kvals, c->slots, d_x, d_rhs,
                                    c->r_batch, c->omega_part, c->stat, c->omega_dev, c->batch, st));
    }
    KKT_CUDA(cudaMemcpyAsync(h_omega, c->omega_dev, sizeof(double) * c->batch, cudaMemcpyDeviceToHost, st));
    return KKT_OK;
}

kkt_status kkt_step_host(kkt_ctx* c, const double* h_vals, const double* h_rhs, double* h_x, double tol,
                         kkt_info* info, void* stream)
{
    if (!c || !h_vals || !h_rhs || !h_x || !(tol >= 0)) return KKT_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    KKT_CUDA(cudaMemcpyAsync(c->stage_vals, h_vals, sizeof(double) * c->nnz * c->batch, cudaMemcpyHostToDevice, st));
    KKT_CUDA(cudaMemcpyAsync(c->stage_b, h_rhs, sizeof(double) * c->n * c->batch, cudaMemcpyHostToDevice, st));
    // x goes to h_x together with the backward error; a second copy only if
    // refinement changed it afterwards
    c->x_early = h_x;
    c->x_early_valid = 0;
    kkt_status r = do_refactor_refine(c, c->stage_vals, c->stage_b, c->stage_x, tol, info, st);
    c->x_early = nullptr;
    if (r != KKT_OK && r != KKT_E_NOCONV) return r;
    if (!c->x_early_valid) {
        KKT_CUDA(cudaMemcpyAsync(h_x, c->stage_x, sizeof(double) * c->n * c->batch, cudaMemcpyDeviceToHost, st));
        KKT_CUDA(cudaStreamSynchronize(st));
    }
    return r;
}

// Fork: every context works on its own stream after the caller's stream
// reaches this point; join: the caller's stream waits for all of them. The
// contexts' graphs then run concurrently on the device.
static kkt_status fork_join(kkt_ctx* const* ctxs, int count, cudaStream_t st,
                            const std::function<kkt_status(int, cudaStream_t)>& body)
{
    cudaEvent_t fork = nullptr;
    KKT_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(fork, st);
    kkt_status res = KKT_OK;
    for (int i = 0; i < count && res == KKT_OK && e == cudaSuccess; ++i) {
        kkt_ctx* c = ctxs[i];
        if (!c->work_stream) e = cudaStreamCreateWithFlags(&c->work_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess && !c->done_event) e = cudaEventCreateWithFlags(&c->done_event, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->work_stream, fork, 0);
        if (e == cudaSuccess) res = body(i, c->work_stream);
        if (e == cudaSuccess && res == KKT_OK) e = cudaEventRecord(c->done_event, c->work_stream);
        if (e == cudaSuccess && res == KKT_OK) e = cudaStreamWaitEvent(st, c->done_event, 0);
    }
    cudaEventDestroy(fork);
    if (e != cudaSuccess) return KKT_E_CUDA;
    return res;
}

kkt_status kkt_refactor_batched(kkt_ctx* const* ctxs, const double* const* d_vals, int count, void* stream)
{
    if (!ctxs || !d_vals || count < 0) return KKT_E_ARG;
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i] || !d_vals[i]) return KKT_E_ARG;
        if (ctxs[i]->opt.precision != ctxs[0]->opt.precision) return KKT_E_ARG;
        for (int j = 0; j < i; ++j) if (ctxs[j] == ctxs[i]) return KKT_E_ARG;
    }
    return fork_join(ctxs, count, (cudaStream_t)stream,
                     [&](int i, cudaStream_t s) { return do_refactor(ctxs[i], d_vals[i], s); });
}

kkt_status kkt_group_create(kkt_ctx* const* ctxs, int count, kkt_group** out)
{
    if (!out || !ctxs || count < 1) return KKT_E_ARG;
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i]) return KKT_E_ARG;
        if (ctxs[i]->opt.precision != ctxs[0]->opt.precision) return KKT_E_ARG;
        for (int j = 0; j < i; ++j) if (ctxs[j] == ctxs[i]) return KKT_E_ARG;
    }
    kkt_group* g = nullptr;
    try {
        g = new kkt_group();
        g->ctxs.assign(ctxs, ctxs + count);
    } catch (...) {
        delete g;
        return KKT_E_NOMEM;
    }
    g->precision = ctxs[0]->opt.precision;
    kkt_status s = g->precision == KKT_FP32_IR ? group_tables<float>(g) : group_tables<double>(g);
    if (s != KKT_OK) {
        kkt_group_destroy(g);
        return s;
    }
    *out = g;
    return KKT_OK;
}

kkt_status kkt_refactor_group(kkt_group* g, const double* const* d_vals, void* stream)
{
    if (!g || !d_vals) return KKT_E_ARG;
    const int count = (int)g->ctxs.size();
    for (int i = 0; i < count; ++i) if (!d_vals[i]) return KKT_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const bool f32 = g->precision == KKT_FP32_IR;
    kkt_status s = fork_join(g->ctxs.data(), count, st, [&](int i, cudaStream_t ws) {
        kkt_ctx* c = g->ctxs[i];
        c->info.status = KKT_OK;
        return f32 ? refactor_levels_t<float>(c, d_vals[i], ws) : refactor_levels_t<double>(c, d_vals[i], ws);
    });
    if (s != KKT_OK) return s;
    if (g->total > 0) {
        kkt_ctx* c0 = g->ctxs[0];
        KKT_CUDA(cudaMemsetAsync(g->gctr, 0, kCtrHead * sizeof(int), st));
        Launch L(c0, st, KK_TREE_FACTOR, 1);
        KKT_CUDA(f32 ? launch_tree_factor_group<float>(static_cast<const TreeJob<float>*>(g->jobs), g->segs, g->nseg,
                                                      g->total, g->gctr, g->spin_limit, g->grid, g->smem, st)
                     : launch_tree_factor_group<double>(static_cast<const TreeJob<double>*>(g->jobs), g->segs,
                                                        g->nseg, g->total, g->gctr, g->spin_limit, g->grid, g->smem,
                                                        st));
    }
    for (kkt_ctx* c : g->ctxs) {
        c->last_vals = c->kvals;
        c->refactored = 1;
        c->refactor_count++;
    }
    return KKT_OK;
}

kkt_status kkt_group_destroy(kkt_group* g)
{
    if (!g) return KKT_OK;
    if (g->dev) cudaFree(g->dev);
    delete g;
    return KKT_OK;
}

kkt_status kkt_solve_batched(kkt_ctx* const* ctxs, const double* const* d_rhs, double* const* d_x, int count,
                             void* stream)
{
    if (!ctxs || !d_rhs || !d_x || count < 0) return KKT_E_ARG;
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i] || !d_rhs[i] || !d_x[i]) return KKT_E_ARG;
        if (!ctxs[i]->refactored) return KKT_E_STATE;
        for (int j = 0; j < i; ++j) if (ctxs[j] == ctxs[i]) return KKT_E_ARG;
    }
    return fork_join(ctxs, count, (cudaStream_t)stream,
                     [&](int i, cudaStream_t s) { return do_solve(ctxs[i], d_rhs[i], d_x[i], s); });
}

kkt_status kkt_residual(kkt_ctx* c, const double* d_rhs, const double* d_x, double* d_r, double* omega_out,
                        void* stream)
{
    if (!c || !d_rhs || !d_x || !d_r) return KKT_E_ARG;
    if (!c->refactored) return KKT_E_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    KKT_CUDA(launch_spmv_resid(c->sched, c->last_vals, d_x, d_rhs, d_r, st));
    if (omega_out) {
        double knorm = 0.0, rm, rs, xm, xs, bm, bs;
        kkt_status s;
        if ((s = knorm_of(c, st, &knorm)) != KKT_OK) return s;
        if ((s = norms_host(c, d_r, &rm, &rs, st)) != KKT_OK) return s;
        if ((s = norms_host(c, d_x, &xm, &xs, st)) != KKT_OK) return s;
        if ((s = norms_host(c, d_rhs, &bm, &bs, st)) != KKT_OK) return s;
        double den = knorm * xm + bm;
        *omega_out = den > 0 ? rm / den : (den == 0 ? rm : den);     // a NaN norm gives NaN
    }
    return KKT_OK;
}

kkt_status kkt_get_info(const kkt_ctx* c, kkt_info* info)
{
    if (!c || !info) return KKT_E_ARG;
    *info = c->info;
    info->refactor_count = c->refactor_count;
    info->launches = c->launches;
    info->batch = c->batch;
    if (c->refactored) {
        DevStat hs;
        KKT_CUDA(cudaDeviceSynchronize());
        KKT_CUDA(cudaMemcpy(&hs, c->stat, sizeof(DevStat), cudaMemcpyDeviceToHost));
        info->n_perturbed = hs.n_perturbed;
        if (hs.numeric_bad) info->status = KKT_E_NUMERIC;
        if (hs.timeout) info->status = KKT_E_TIMEOUT;
    }
    return KKT_OK;
}

int kkt_kernel_stats(kkt_ctx* c, kkt_kernel_stat* out, int max_out)
{
    if (!c || !out || max_out <= 0) return -1;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    double ms[KK_COUNT] = {0};
    long long cnt[KK_COUNT] = {0};
    for (size_t slot = 0; slot < c->ev_used / 2; ++slot) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, c->ev[2 * slot], c->ev[2 * slot + 1]) != cudaSuccess) continue;
        ms[c->ev_kind[slot]] += t;
        cnt[c->ev_kind[slot]] += c->ev_count[slot];
    }
    c->ev_used = 0;
    int k = 0;
    for (int i = 0; i < KK_COUNT && k < max_out; ++i) {
        if (!cnt[i]) continue;
        out[k].name = kKernelNames[i];
        out[k].launches = cnt[i];
        out[k].ms = ms[i];
        ++k;
    }
    return k;
}

kkt_status kkt_set_profiling(kkt_ctx* c, int on)
{
    if (!c) return KKT_E_ARG;
    c->profile = on ? 1 : 0;
    c->ev_used = 0;
    return KKT_OK;
}

kkt_status kkt_get_plan(const kkt_ctx* c, kkt_plan_info* out)
{
    if (!c || !out) return KKT_E_ARG;
    const Analysis& an = c->an;
    std::memset(out, 0, sizeof(*out));
    out->n = c->n;
    out->nnz = an.nnz;
    out->nnz_lu = an.nnz_l + an.nnz_u;
    out->stored_factor = an.stored_factor;
    out->n_fronts = an.ns;
    out->n_levels = an.n_levels;
    out->max_front = an.max_front;
    out->max_pivots = an.max_pivots;
    out->flops = an.flops;
    out->flops_exact = an.flops_exact;
    out->device_bytes = c->device_bytes;
    out->batch = c->batch;
    out->tree_levels = an.n_levels - c->tree_split;
    out->tree_units = c->tsched.nunits;
    out->tree_bytes = c->tree_bytes;
    out->tree_nnz_k = c->tree_nnz_k;
    out->tree_nnz_lu = c->tree_nnz_lu;
    out->tree_pivots = c->tree_pivots;
    return KKT_OK;
}

kkt_status kkt_debug_stall(kkt_ctx* c)
{
    if (!c) return KKT_E_ARG;
    if (c->tsched.nq == 0) return KKT_E_STATE;
    const int req[2] = {1, 0};
    KKT_CUDA(cudaDeviceSynchronize());
    KKT_CUDA(cudaMemcpy(c->stall, req, sizeof(req), cudaMemcpyHostToDevice));
    KKT_CUDA(cudaDeviceSynchronize());                    // landed before any later launch, on any stream
    return KKT_OK;
}

kkt_status kkt_debug_pivot_rcp(const void* d_in, void* d_out, int64_t n, int precision, void* stream)
{
    if (n < 0 || (precision != KKT_FP64 && precision != KKT_FP32_IR)) return KKT_E_ARG;
    if (n == 0) return KKT_OK;
    if (!d_in || !d_out || (n + 255) / 256 > 0x7fffffff) return KKT_E_ARG;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == KKT_FP64)
        pivot_rcp_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(d_in),
                                                         static_cast<double*>(d_out), n);
    else
        pivot_rcp_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(d_in),
                                                        static_cast<float*>(d_out), n);
    KKT_CUDA(cudaGetLastError());
    return KKT_OK;
}

kkt_status kkt_get_perm(const kkt_ctx* c, int32_t* h_perm)
{
    if (!c || !h_perm) return KKT_E_ARG;
    std::memcpy(h_perm, c->an.perm.data(), sizeof(int32_t) * c->n);
    return KKT_OK;
}

kkt_status kkt_get_scaling(const kkt_ctx* c, double* h_d)
{
    if (!c || !h_d) return KKT_E_ARG;
    if (!c->refactored) return KKT_E_STATE;
    KKT_CUDA(cudaDeviceSynchronize());
    KKT_CUDA(cudaMemcpy(h_d, c->d_final, sizeof(double) * c->n, cudaMemcpyDeviceToHost));
    return KKT_OK;
}

kkt_status kkt_export_factors(const kkt_ctx* c, int64_t* nl, int32_t* l_row, int32_t* l_col, double* l_val,
                              int64_t* nu, int32_t* u_row, int32_t* u_col, double* u_val)
{
    if (!c || !nl || !nu) return KKT_E_ARG;
    const Analysis& an = c->an;
    int64_t cl = 0, cu = 0;
    for (int s = 0; s < an.ns; ++s) {
        int64_t w = an.sn_first[s + 1] - an.sn_first[s], F = an.sn_front[s];
        cl += w * (w - 1) / 2 + (F - w) * w;
        cu += w * (w + 1) / 2 + w * (F - w);
    }
    *nl = cl;
    *nu = cu;
    if (!l_row && !u_row) return KKT_OK;
    if (!l_row || !l_col || !l_val || !u_row || !u_col || !u_val) return KKT_E_ARG;
    if (!c->refactored) return KKT_E_STATE;
    const size_t es = elem_size(c->opt.precision);
    std::vector<char> host((size_t)an.panel_total * es);
    const void* src = c->opt.precision == KKT_FP32_IR ? (const void*)c->nf.panel : (const void*)c->nd.panel;
    KKT_CUDA(cudaDeviceSynchronize());
    KKT_CUDA(cudaMemcpy(host.data(), src, host.size(), cudaMemcpyDeviceToHost));
    auto val = [&](int64_t idx) -> double {
        if (es == 4) return (double)reinterpret_cast<const float*>(host.data())[idx];
        return reinterpret_cast<const double*>(host.data())[idx];
    };
    int64_t il = 0, iu = 0;
    for (int s = 0; s < an.ns; ++s) {
        int w = an.sn_first[s + 1] - an.sn_first[s], F = an.sn_front[s];
        const int* R = an.rows.data() + an.rows_ptr[s];
        int64_t off = an.panel_off[s];
        for (int b = 0; b < w; ++b)
            for (int a = 0; a < F; ++a) {
                double v = val(off + a + (int64_t)b * F);
                int r = an.perm[R[a]], col = an.perm[R[b]];
                if (a > b) { l_row[il] = r; l_col[il] = col; l_val[il] = v; ++il; }
                else { u_row[iu] = r; u_col[iu] = col; u_val[iu] = v; ++iu; }
            }
        int m = F - w;
        for (int a = 0; a < w; ++a)
            for (int b = 0; b < m; ++b) {
                double v = val(off + (int64_t)F * w + a + (int64_t)b * w);
                u_row[iu] = an.perm[R[a]]; u_col[iu] = an.perm[R[w + b]]; u_val[iu] = v; ++iu;
            }
    }
    return KKT_OK;
}

kkt_status kkt_destroy(kkt_ctx* c)
{
    if (!c) return KKT_OK;
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->g_factor) cudaGraphExecDestroy(c->g_factor);
    if (c->g_solve) cudaGraphExecDestroy(c->g_solve);
    if (c->g_ffwd) cudaGraphExecDestroy(c->g_ffwd);
    if (c->g_bwd) cudaGraphExecDestroy(c->g_bwd);
    if (c->g_levels) cudaGraphExecDestroy(c->g_levels);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->work_stream) cudaStreamDestroy(c->work_stream);
    if (c->done_event) cudaEventDestroy(c->done_event);
    if (c->pool.base) cudaFree(c->pool.base);
    if (c->pin) cudaFreeHost(c->pin);
    if (c->stat_pin) cudaFreeHost(c->stat_pin);
    delete c;
    return KKT_OK;
}

}  // extern "C"
