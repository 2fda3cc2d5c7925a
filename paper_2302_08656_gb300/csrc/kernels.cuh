// Device data layout and kernel launchers of the GB300 KKT path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kktgb {

// Read-only schedule produced by the host analysis, resident in HBM.
struct DevSched {
    int n = 0;
    int64_t nnz = 0;
    int ns = 0;
    const int* rowptr = nullptr;      // K pattern (n+1)
    const int* colidx = nullptr;      // (nnz)
    const int* perm = nullptr;        // step -> original index (n)
    const int* sn_first = nullptr;    // (ns+1)
    const int* sn_front = nullptr;    // (ns)
    const int64_t* rows_ptr = nullptr;
    const int* rows = nullptr;
    const int* child_ptr = nullptr;
    const int* child_list = nullptr;
    const int64_t* asm_ptr = nullptr;
    const int* asm_pos = nullptr;
    const int* asm_src = nullptr;
    const int64_t* rel_ptr = nullptr;
    const int* rel = nullptr;
    const int64_t* panel_off = nullptr;
    const int64_t* cb_off = nullptr;
    const int* cb_split = nullptr;    // per front: contribution rows landing on parent pivots
    const int64_t* inv_off = nullptr; // per panel-class front: offset of its children's gather maps
    const int* inv = nullptr;         // per (front, child): parent CB row -> child CB row or -1
    const int64_t* f12_off = nullptr; // per panel-class front: offset of its assembled pivot rows
    // sliced ELLPACK copy of K's pattern (SellPlan): per-refactor copies of K
    // and D K D are stored in this layout; asm_src indexes it
    int nslices = 0;
    int64_t slots = 0;
    const int64_t* sell_off = nullptr;    // nslices + 1
    const int* sell_row = nullptr;        // nslices * 32 (-1: no row)
    const int* sell_ci = nullptr;         // slots (-1: padding)
    const int* sell_src = nullptr;        // slots: CSR position (-1: padding)
};

// Device-side counters of one context, cleared at the start of each refactor.
struct DevStat {
    unsigned long long amax_bits;     // max |D K D| as the bits of a non-negative double
    unsigned long long knorm_bits;    // ||K||_inf
    int n_perturbed;
    int numeric_bad;
    int ruiz_changed[64];
    int timeout;                      // a bounded wait of a tree kernel gave up
};

// Per-context numeric buffers.
template <typename T>
struct DevNum {
    const double* vals = nullptr;     // K values of the current refactor (caller memory, CSR order)
    double* kcopy = nullptr;          // library-owned copy of K in the sliced layout (residuals use it)
    unsigned short* keys = nullptr;   // per slot: exponent key of |k| (equilibration passes)
    double* d = nullptr;              // equilibration factors (n)
    double* dtmp = nullptr;           // ping-pong buffer (n)
    T* sv = nullptr;                  // D K D in factor precision (sliced layout, slots)
    T* panel = nullptr;               // factor panels
    T* cb = nullptr;                  // contribution blocks
    T* vec = nullptr;                 // step-space solve vector (n)
    T* cbv = nullptr;                 // solve contribution vectors
    T* f12 = nullptr;                 // assembled pivot rows of panel-class fronts
    DevStat* stat = nullptr;
    double pivot_eps = 1e-14;
    // element strides between consecutive instances of a batch (0 for one instance)
    int64_t bs_nnz = 0, bs_slot = 0, bs_n = 0, bs_panel = 0, bs_cb = 0, bs_cbv = 0, bs_f12 = 0;
    __host__ __device__ DevNum at(int b) const
    {
        DevNum r = *this;
        if (b) {
            r.vals += b * bs_nnz;
            r.kcopy += b * bs_slot;
            r.keys += b * bs_slot;
            r.d += b * bs_n;
            r.dtmp += b * bs_n;
            r.sv += b * bs_slot;
            r.panel += b * bs_panel;
            r.cb += b * bs_cb;
            r.vec += b * bs_n;
            r.cbv += b * bs_cbv;
            r.f12 += b * bs_f12;
            r.stat += b;
        }
        return r;
    }
};

// Reciprocal of a pivot, 1 / d within one unit in the last place, used by
// every kernel that needs 1 / u_pp (factorization and backward solves alike,
// so all schedules stay bitwise equal). Newton-Raphson from the hardware
// approximation x0 (rcp.approx.ftz): with e = 1 - d x0, formed exactly by an
// FMA, 1 / d = x0 / (1 - e) = x0 (1 + e + e^2 + ...). Double precision takes
// the series to e^2, x1 = x0 + x0 (e + e^2), relative error about e^3 plus
// the last rounding (|e| < 2^-19 measured on GB300: e^3 < 2^-57); single
// precision takes x1 = x0 + x0 e (error about e^2). Three dependent FP64 FMAs
// against the longer IEEE division, on the critical path of every pivot.
// Outside [2^-1000, 2^1000] (2^-100, 2^100 in single precision), for zero,
// infinities and NaN the IEEE division is used, so the approximation never
// meets a flushed subnormal.
#ifdef __CUDACC__
// pivot_rcp_fast is the Newton step alone and pivot_rcp_fast_ok tells whether
// it is pivot_rcp's answer (d inside the range above): a caller on a critical
// path takes the fast value at once, tests the range off that path and
// repeats the work with pivot_rcp in the rare case it fails.
__device__ __forceinline__ bool pivot_rcp_fast_ok(double d)
{
    return ((((unsigned)(__double_as_longlong(d) >> 52)) & 0x7ffu) - 23u) <= 2000u;
}
__device__ __forceinline__ double pivot_rcp_fast(double d)
{
    double x0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x0) : "d"(d));
    const double e = fma(-d, x0, 1.0);
    return fma(x0, fma(e, e, e), x0);
}
__device__ __forceinline__ double pivot_rcp(double d)
{
    if (!pivot_rcp_fast_ok(d)) return 1.0 / d;
    return pivot_rcp_fast(d);
}
__device__ __forceinline__ bool pivot_rcp_fast_ok(float d)
{
    return (((__float_as_uint(d) >> 23) & 0xffu) - 27u) <= 200u;
}
__device__ __forceinline__ float pivot_rcp_fast(float d)
{
    float x0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x0) : "f"(d));
    return fmaf(x0, fmaf(-d, x0, 1.0f), x0);
}
__device__ __forceinline__ float pivot_rcp(float d)
{
    if (!pivot_rcp_fast_ok(d)) return 1.0f / d;
    return pivot_rcp_fast(d);
}
#endif

// Static pivoting, on the bit patterns (integer pipes only: FP64 compares
// have long latency on this GPU and sit on the critical path of every pivot):
// a pivot with |piv| < floorT (floorT >= 0, in the factor precision) is
// replaced by sign(piv) * floorT (sign(0) = +1) and counted; NaN/Inf raise
// the flag and are returned unchanged.
#ifdef __CUDACC__
__device__ __forceinline__ double static_pivot(double piv, double floorT, DevStat* stat, bool count)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(piv);
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    if (mag >= 0x7ff0000000000000ull) {
        if (count) atomicExch(&stat->numeric_bad, 1);
        return piv;
    }
    const unsigned long long fb = (unsigned long long)__double_as_longlong(floorT);
    if (mag < fb && fb < 0x7ff0000000000000ull) {
        if (count) atomicAdd(&stat->n_perturbed, 1);
        return __longlong_as_double((long long)(fb | (mag ? (b & 0x8000000000000000ull) : 0ull)));
    }
    return piv;
}
__device__ __forceinline__ float static_pivot(float piv, float floorT, DevStat* stat, bool count)
{
    const unsigned b = __float_as_uint(piv);
    const unsigned mag = b & 0x7fffffffu;
    if (mag >= 0x7f800000u) {
        if (count) atomicExch(&stat->numeric_bad, 1);
        return piv;
    }
    const unsigned fb = __float_as_uint(floorT);
    if (mag < fb && fb < 0x7f800000u) {
        if (count) atomicAdd(&stat->n_perturbed, 1);
        return __uint_as_float(fb | (mag ? (b & 0x80000000u) : 0u));
    }
    return piv;
}
// The same decision without branches or atomics, for a warp that computes the
// pivot uniformly (every lane the same value): the events are returned in
// bad / pert and counted once by the caller.
__device__ __forceinline__ float static_pivot_sel(float piv, float floorT, bool& bad, bool& pert)
{
    const unsigned b = __float_as_uint(piv);
    const unsigned mag = b & 0x7fffffffu;
    const unsigned fb = __float_as_uint(floorT);
    bad = mag >= 0x7f800000u;
    pert = !bad && mag < fb && fb < 0x7f800000u;
    return pert ? __uint_as_float(fb | (mag ? (b & 0x80000000u) : 0u)) : piv;
}
__device__ __forceinline__ double static_pivot_sel(double piv, double floorT, bool& bad, bool& pert)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(piv);
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    const unsigned long long fb = (unsigned long long)__double_as_longlong(floorT);
    bad = mag >= 0x7ff0000000000000ull;
    pert = !bad && mag < fb && fb < 0x7ff0000000000000ull;
    return pert ? __longlong_as_double((long long)(fb | (mag ? (b & 0x8000000000000000ull) : 0ull))) : piv;
}
#endif

// One launch group: the fronts of one level of one context.
struct FrontTile { int front; int ti; int tj; };

constexpr int kWarpFrontMax = 32;      // fronts with F <= 32 are handled by one warp
constexpr int kWarpStageV = 512;       // per warp: staged child-block values, at most
constexpr int kWarpStageR = 192;       // ... and staged relative indices
constexpr int kWarpLevelMin = 608;     // ... when their level has at least 4 x 152 of them
constexpr int kPanelCbMin = 32;        // fronts with F - w >= 32 use panel + tiled Schur update
constexpr int kTile = 16;              // Schur update tile (kTile x kTile)
constexpr int kSeqSum = 32;            // backward solve: U12 x summed in sequence up to this many terms

// ---- narrow top of the assembly tree: persistent, dependency-driven kernels
//
// Levels from `split` upward (those with few fronts) are not launched level by
// level: one persistent kernel per phase takes work units in dependency order
// from an atomic ticket counter; a unit waits (bounded) until the units it
// depends on have signalled completion, then runs. Every front of this part
// is factored as nt x nt units; unit (ti, tj) eliminates the w pivots of the
// "mini front" made of the pivot rows/columns and the ts-row (ts-column)
// stripe ti (tj) of the contribution block: all units of a front repeat the
// factorization of the pivot block (identical data, identical result) and
// each produces its own tile of L21, U12 and the contribution block.
struct TreeFront {
    int f, first, w, F;          // supernode, first pivot step, pivots, front order
    int ts, nt;                  // tile size and tiles per dimension of the contribution block
    int kid_begin, kid_end;      // children (TreeKid range)
    int parent;                  // tree index of the parent front, -1 at a root
    int units;                   // nt * nt
    int64_t asm_begin, asm_end;  // original entries (Analysis asm lists)
    int64_t panel_off, cb_off, rel_ptr, rows_ptr;
    int64_t inv_off;             // gather maps: child c (local) at inv_off + c * (F - w)
};
// A work unit of the tree kernels with its front's descriptor, read by a CTA
// in one step.
struct TreeUnit {
    TreeFront d;
    FrontTile u;
    int pad;
};
struct TreeKid {
    int q;                       // tree index of the child, -1 if the child lies below the tree part
    int mc, k;                   // child contribution-block order; its rows landing on parent pivots
    int units;                   // units of the child (0 below the tree part)
    int64_t cb_off, rel_ptr;
};
struct TreeSched {
    int nq = 0;                  // fronts of the tree part (tree index = level-major order)
    int nunits = 0;              // factorization units
    const TreeFront* fr = nullptr;
    const TreeKid* kid = nullptr;
    const TreeUnit* unit = nullptr;    // factorization units in dependency order (front = tree index)
    const TreeUnit* unit_fused = nullptr;   // the same with a forward-solve unit (ti = -1) per front after its level
    int nunits_fused = 0;
    size_t kid_off = 0;                // shared-memory offset of the children's descriptors (factor kernel)
    const int* inv = nullptr;          // gather maps: parent CB row -> child CB row or -1
    // shared-memory layout parameters (host computed)
    int max_kids = 0, map_w = 0, m_elems = 0;
    int max_F = 0, max_w = 0;
    int fwd_stage = 0;           // 1: forward solve stages the F x w panel in shared memory
    int bwd_stage = 0;           // 1: backward solve stages U12 in shared memory
    int fwd_cstage = 0;          // 1: forward solve by chains stages two F x w panels (else pivot blocks)
    int fwd_kstage = 0;          // children's contribution entries staged per front by the forward chains
    int max_fw = 0, max_wm = 0;
    // backward substitution by chains: chain c is the fronts bwd_chain[bwd_chain_ptr[c] ..
    // bwd_chain_ptr[c + 1] - 1], top first, each the only tree child of the one before
    const int* bwd_chain = nullptr;
    const int* bwd_chain_ptr = nullptr;
    int nchains = 0;
};
// One context of a group whose tree parts run in one launch (see
// tree_factor_kernel): its schedule, numeric buffers, instances and counter
// block; and the segments of the group's ticket space: tickets start ..
// (next start) - 1 are units ul0, ul0 + 1, ... (times the context's
// instances) of context `job`.
template <typename T>
struct TreeJob {
    DevSched s;
    TreeSched ts;
    DevNum<T> nm;
    int B = 1;
    int* ctr = nullptr;
};
struct TreeSeg {
    int start;
    int job;
    int ul0;
};

constexpr int kTreeMaxKids = 48;       // fronts with more children stay level-launched
constexpr int kTreeStage = 2048;       // staged child contribution entries per pass (forward solve)
// Counter block of a tree kernel: [0] ticket, [1] abort flag, [2] forward-solve ticket
// (solve block), [3] backward-solve ticket; then the per-(instance, front) completion counters.
constexpr int kCtrHead = 4;

// Launchers (all asynchronous on `st`).
// Equilibration: iteration 0 copies K (caller's CSR values, instance stride
// bs_nnz) into the sliced copy kcopy with its exponent keys (stride bs_slot);
// iters = 0 makes only that copy and sets d = 1.
cudaError_t launch_ruiz(const DevSched& s, const double* vals, int64_t bs_nnz, double* kcopy, unsigned short* keys,
                        int64_t bs_slot, double* d, double* dtmp, int iters, DevStat* stat, double** d_final,
                        int batch, cudaStream_t st);
template <typename T>
cudaError_t launch_scale(const DevSched& s, const DevNum<T>& nm, const double* d, int batch, cudaStream_t st);
template <typename T>
cudaError_t launch_fronts_warp(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count,
                               int max_front, int stage_v, int stage_r, int fused, int batch, cudaStream_t st);
template <typename T>
cudaError_t launch_fronts_leaf(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, int group,
                               int fused, int batch, cudaStream_t st);
template <typename T>
cudaError_t launch_solve_bwd_leaf(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, int group,
                                  int batch, cudaStream_t st);
template <typename T>
cudaError_t launch_fronts_cta(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count,
                              int max_front, int batch, cudaStream_t st);
template <typename T>
cudaError_t launch_fronts_panel(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count,
                                size_t smem_bytes, T* gscratch, int64_t scratch_stride, int batch, cudaStream_t st);
template <typename T>
cudaError_t launch_schur_tiles(const DevSched& s, const DevNum<T>& nm, const FrontTile* tiles, int count,
                               int max_w, int batch, cudaStream_t st);
template <typename T>
cudaError_t launch_solve_fwd_cta(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count,
                                 int max_front, int max_w, int batch, cudaStream_t st);
template <typename T>
cudaError_t launch_solve_bwd_cta(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count,
                                 int max_front, int max_w, int batch, cudaStream_t st);
template <typename T>
cudaError_t launch_solve_pre(const DevSched& s, const DevNum<T>& nm, const double* b, int batch, cudaStream_t st);
template <typename T>
cudaError_t launch_solve_fwd(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count,
                             int max_front, int max_w, int batch, cudaStream_t st);
template <typename T>
cudaError_t launch_solve_bwd(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count,
                             int max_front, int max_w, int batch, cudaStream_t st);
template <typename T>
cudaError_t launch_solve_post(const DevSched& s, const DevNum<T>& nm, double* x, int batch, cudaStream_t st);
// per instance: r = b - K x, omega = ||r||_inf / (||K||_inf ||x||_inf + ||b||_inf) into omega[b],
// K the sliced copy (instance stride bs_slot); part holds batch * resid_blocks(n) * 4 doubles
constexpr int kResidRows = 64;         // rows per block of the partial-maxima buffer (an upper bound)
inline int resid_blocks(int n) { return (n + kResidRows - 1) / kResidRows; }
// ||K||_inf of every instance is read from stat[inst].knorm_bits (the refactorization's scaling pass)
cudaError_t launch_resid_omega(const DevSched& s, const double* kvals, int64_t bs_slot, const double* x,
                               const double* b, double* r, double* part, const DevStat* stat, double* omega,
                               int batch, cudaStream_t st);

// FP64 vector kernels for the residual and FGMRES (kv: one instance's sliced copy of K).
cudaError_t launch_spmv_resid(const DevSched& s, const double* kv, const double* x, const double* b, double* r,
                              cudaStream_t st);
cudaError_t launch_spmv(const DevSched& s, const double* kv, const double* x, double* y, cudaStream_t st);
// FGMRES's small work on the device: Arnoldi step j (Hessenberg column, Givens
// rotations, g, convergence flag), the start of a cycle, the least-squares solve
cudaError_t launch_fgmres_givens(int j, int ldh, const double* h2, const double* nrm, double* H, double* cs,
                                 double* sn, double* g, double* scale, double* flag, double target, cudaStream_t st);
cudaError_t launch_fgmres_start(int m, double beta, double* g, double* scale, cudaStream_t st);
cudaError_t launch_fgmres_lsq(int k, int ldh, const double* H, const double* g, double* y, cudaStream_t st);
// out[k] = <V_k, w> for k < nv (V column-major with leading dimension ldv); out zeroed inside
cudaError_t launch_multidot(int n, const double* V, int64_t ldv, int nv, const double* w, double* out,
                            cudaStream_t st);
// w -= V * h (nv columns)
cudaError_t launch_multiaxpy(int n, double* w, const double* V, int64_t ldv, int nv, const double* h,
                             cudaStream_t st);
// y = alpha * x (alpha from device pointer, inverted if invert != 0)
cudaError_t launch_scal_copy(int n, const double* x, double* y, const double* alpha, int invert,
                             cudaStream_t st);
// x += Z * y (nv columns)
cudaError_t launch_update(int n, double* x, const double* Z, int64_t ldz, int nv, const double* y,
                          cudaStream_t st);
// out[0] = max |a|, out[1] = sum a^2 (zeroed inside); for several vectors in one launch
cudaError_t launch_norms(int n, const double* a, double* out, cudaStream_t st);
cudaError_t launch_zero_stat(DevStat* stat, cudaStream_t st);

// Tree kernels. grid = persistent CTAs; ctr = counter block (zeroed by the
// caller before the launch); stall = optional test hook (see kkt_debug_stall).
template <typename T>
cudaError_t tree_grid(int kind, size_t smem, int* grid);   // kind 0 factor, 1 forward, 2 backward
// fused != 0: the factor kernel also runs the forward substitution of every tree front (its counter
// block then holds batch * nq factor counters followed by batch * nq forward counters)
// The tree parts of a group of contexts in one launch; gctr: the group's
// counter block (ticket, abort flag), cleared by the caller.
template <typename T>
cudaError_t launch_tree_factor_group(const TreeJob<T>* jobs, const TreeSeg* segs, int nseg, int total, int* gctr,
                                     long long spin_limit, int grid, size_t smem, cudaStream_t st);
template <typename T>
cudaError_t launch_tree_factor(const DevSched& s, const TreeSched& t, const DevNum<T>& nm, int batch, int* ctr,
                               int* stall, long long spin_limit, int grid, size_t smem, int fused, int u0, int nu,
                               int tick, cudaStream_t st);
template <typename T>
cudaError_t launch_tree_fwd(const DevSched& s, const TreeSched& t, const DevNum<T>& nm, int batch, int* ctr,
                            long long spin_limit, int grid, size_t smem, cudaStream_t st);
template <typename T>
cudaError_t launch_tree_bwd(const DevSched& s, const TreeSched& t, const DevNum<T>& nm, int batch, int* ctr,
                            long long spin_limit, int grid, size_t smem, cudaStream_t st);
cudaError_t configure_tree_kernels(int optin);

// Jacobi-sweep preconditioner (jacobi.cu): `sweeps` sweeps with L then U on
// the step-space vector nm.vec, result in nm.vec; lptr / lidx: per step row,
// the contribution-vector offsets of the descendant fronts' L21 rows.
template <typename T>
cudaError_t launch_jacobi(const DevSched& s, const DevNum<T>& nm, int sweeps, bool block, const int* lptr, const int* lidx,
                          T* ya, T* yb, T* xa, T* t, int* launches, cudaStream_t st);

}  // namespace kktgb
