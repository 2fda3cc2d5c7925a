// Persistent, dependency-driven kernels for the narrow top of the assembly
// tree (refactorization, forward and backward substitution).
//
// Above a few hundred fronts per level the per-level launches of the
// multifrontal refactorization (Alg. 1 refactor step) and of the triangular
// solves are bound by latency: one CTA per front spends its time on chains of
// dependent loads and on the launch boundary between levels. Here the whole
// narrow part of the tree is one launch per phase. Work units are numbered in
// a dependency order (level-major); CTAs take them from an atomic ticket
// counter, load everything that does not depend on other units (descriptors,
// original entries, gather maps, factor panels), then wait -- bounded, with
// an error flag on expiry -- until the units they depend on have signalled
// completion, and finish with the data those units produced.
//
// Forward progress: a CTA holding ticket t only waits for units with smaller
// tickets, which are already held by running CTAs; by induction the smallest
// unfinished ticket can always run, whatever the residency of the grid.
//
// Every entry is computed with the same operations in the same order as the
// level-launched kernels (assembly: original entry, then the children in
// order; elimination: updates in pivot order, one reciprocal per pivot), so
// both paths give bitwise identical factors and solutions.
#include "kernels.cuh"

#include <algorithm>
#include <cstdlib>

namespace kktgb {

namespace {

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until *p >= need, at most `limit` polls. Returns false if the wait
// gave up or another CTA aborted the kernel; on expiry the abort flag is set.
__device__ bool bounded_wait(const int* p, int need, int* abort_flag, long long limit)
{
    long long it = 0;
    while (ld_acquire(p) < need) {
        if (ld_acquire(abort_flag)) return false;
        if (++it > limit) {
            atomicExch(abort_flag, 1);
            return false;
        }
        __nanosleep(100);
    }
    return true;
}

// Bounded wait of warp 0 for the children of a unit: lane l polls the
// completion counters of children l, l + 32, ... (need = their unit count,
// or 1 if `one`), so every child is checked in each round while the other
// warps of the CTA stay parked at the next barrier. Returns 1 once all are
// complete, 0 if the wait gave up (the abort flag is then set) or another CTA
// aborted the kernel. Called by warp 0 only.
__device__ int warp_wait_kids(const int* done_b, const TreeKid* kids, int nk, bool one, int* abort_flag,
                              long long limit, const int* extra = nullptr, int extra_need = 0)
{
    const int lane = threadIdx.x & 31;
    for (long long it = 0;; ++it) {
        bool ok = true;
        for (int c = lane; c < nk; c += 32)
            if (kids[c].q >= 0 && ld_acquire(done_b + kids[c].q) < (one ? 1 : kids[c].units)) ok = false;
        if (extra && lane == 0 && ld_acquire(extra) < extra_need) ok = false;
        if (__all_sync(0xffffffffu, ok)) return 1;
        if ((it & 31) == 31) {
            int stop = 0;
            if (lane == 0) {
                stop = ld_acquire(abort_flag);
                if (!stop && it > limit) {
                    atomicExch(abort_flag, 1);
                    stop = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, stop, 0)) return 0;
        }
        __nanosleep(64);
    }
}

// Signal completion of a unit: after a CTA barrier (every thread's stores
// happen before it), one thread adds 1 to the counter with a release
// reduction at GPU scope, which makes them visible to a CTA that acquires the
// counter.
__device__ __forceinline__ void signal_done(int* counter)
{
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(counter) : "memory");
}

// Take the next ticket (or `total` once the kernel was aborted): the abort
// flag and the ticket counter are read together, in one round trip.
__device__ __forceinline__ int next_ticket(int* ticket, const int* abort_flag, int total, int* s_t)
{
    if (threadIdx.x == 0) {
        int stop;
        asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(stop) : "l"(abort_flag) : "memory");
        const int t = atomicAdd(ticket, 1);
        *s_t = stop ? total : t;
    }
    __syncthreads();
    return *s_t;
}

constexpr int kTreeCtasPerSm = 4;

__host__ __device__ __forceinline__ size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename X>
__device__ __forceinline__ void copy_words(X* dst, const X* src, int count, int tid, int nt)
{
    static_assert(sizeof(X) % 4 == 0, "word copy");
    const int words = count * (int)(sizeof(X) / 4);
    for (int e = tid; e < words; e += nt)
        reinterpret_cast<int*>(dst)[e] = reinterpret_cast<const int*>(src)[e];
}

template <typename T, int NT>
__device__ bool fwd_unit(const DevSched& s, const TreeSched& ts, const DevNum<T>& nm, const TreeFront& d, int q,
                         TreeKid* kids, int* s_cut, int* s_ok, unsigned char* smraw, int* done_b,
                         const int* fac_done, int* abort_flag, long long limit);

// Panel step of the single-precision elimination: warp 0, lane -> row p0 +
// lane, a[k] = column p0 + k of the panel (pk <= 8 active columns), loaded
// from M. Pivot k is computed by every lane from lane k's entry (a shuffle,
// then the static pivot and the reciprocal: the same values on every lane,
// so nothing diverges) and its events are counted once, in bad / pert. FAST:
// the reciprocal's Newton step without its range test; returns false if a
// pivot fell outside that range (the caller then repeats the panel with the
// full pivot_rcp, from the same entries of M). FULL: all 8 columns active
// (pk = 8). Every entry gets the operations of the one-pivot schedule in pivot
// order.
template <bool FAST, bool FULL>
__device__ __forceinline__ bool panel_f32(const float* M, int Fr, int p0, int pk, int row, float floorT, float (&a)[8],
                                          int& bad, int& pert)
{
    const int tx = threadIdx.x & 31;
    bool ok = true;
    bad = 0;
    pert = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = ((FULL || k < pk) && row < Fr) ? M[row + (p0 + k) * Fr] : 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const bool act = FULL || k < pk;                           // warp-uniform
        float u[8];
#pragma unroll
        for (int kk = k + 1; kk < 8; ++kk) u[kk] = __shfl_sync(0xffffffffu, a[kk], k);   // pivot row p0 + k
        const float x = __shfl_sync(0xffffffffu, a[k], k);
        bool b1, p1;
        const float piv = static_pivot_sel(x, floorT, b1, p1);
        float r;
        if (FAST) {
            r = pivot_rcp_fast(piv);
            ok = ok && (!act || pivot_rcp_fast_ok(piv));
        } else {
            r = pivot_rcp(piv);
        }
        if (act) {
            bad |= (int)b1;
            pert += (int)p1;
        }
        const bool lk = act && tx == k, below = act && tx > k;
        a[k] = lk ? piv : (below ? a[k] * r : a[k]);               // l below the pivot
#pragma unroll
        for (int kk = k + 1; kk < 8; ++kk)
            if (below) a[kk] -= a[k] * u[kk];
    }
    return ok;
}

// One kPanel = 8 step of the single-precision elimination of a mini front M
// (Fr x Fc <= 32 x 32, ld Fr) by 256 threads (32 x 8: lane -> row, warp ->
// column group): warp 0 factors the panel (pivot columns p0 .. p0 + pk - 1,
// lane -> row p0 + lane) in registers without a CTA barrier; then every warp
// applies it to its trailing columns j = p0 + pk + warp + 8 c (lane -> row,
// one shuffle per pivot for the row's U entry, its three columns
// interleaved). Each entry still receives its updates in pivot order with
// the same roundings as the one-pivot schedule. FULL: pk = 8.
template <bool FULL>
__device__ __forceinline__ void elim_step_f32(float* M, int Fr, int Fc, int p0, int pk, float floorT, int& n_bad,
                                              int& n_pert)
{
    constexpr int kPanel = 8;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int row = p0 + tx;
    if (ty == 0) {
        float a[kPanel];
        int pb = 0, pp = 0;
        if (!panel_f32<true, FULL>(M, Fr, p0, pk, row, floorT, a, pb, pp))
            panel_f32<false, FULL>(M, Fr, p0, pk, row, floorT, a, pb, pp);   // a reciprocal out of range
        n_bad |= pb;
        n_pert += pp;
        if (row < Fr)
#pragma unroll
            for (int k = 0; k < kPanel; ++k)
                if (FULL || k < pk) M[row + (p0 + k) * Fr] = a[k];
    }
    __syncthreads();
    float lp[kPanel];
#pragma unroll
    for (int k = 0; k < kPanel; ++k) lp[k] = ((FULL || k < pk) && row < Fr) ? M[row + (p0 + k) * Fr] : 0.0f;
    for (int jb = p0 + pk + ty; jb < Fc; jb += 24) {
        float v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = (row < Fr && jb + 8 * c < Fc) ? M[row + (jb + 8 * c) * Fr] : 0.0f;
#pragma unroll
        for (int k = 0; k < kPanel; ++k) {
            const bool upd = (FULL || k < pk) && tx > k;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float u = __shfl_sync(0xffffffffu, v[c], k);   // row p0 + k: final at step k
                if (upd) v[c] -= lp[k] * u;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (row < Fr && jb + 8 * c < Fc) M[row + (jb + 8 * c) * Fr] = v[c];
    }
    __syncthreads();
}

// ------------------------------------------------------------- refactor

// Unit (q, ti, tj) of instance b. Mini front M (Fr x Fc, column-major, ld Fr):
// rows 0..w-1 / columns 0..w-1 are the pivots, rows w..Fr-1 the contribution
// rows i0..i0+nr-1, columns w..Fc-1 the contribution columns j0..j0+nc-1.
// Threads form a 32 x 8 grid (lane -> row, warp -> column).
//
// MULTI: the tree parts of several contexts (patterns of different sizes,
// each possibly batched) in one launch. Tickets 0 .. nu - 1 run through
// segments (one per level of one context, ordered by height below that
// context's root, the highest first, so that the tops of all trees finish
// together); ticket t of segment g is unit ul0 + (t - start) / B, instance
// (t - start) % B of context job: within a context the order is the
// single-context order, so every unit still waits only for smaller tickets.
// Tickets and the abort flag come from the group's counter block (ctr);
// completion counters are each context's own. The descriptors of the current
// unit's context are cached in shared memory.
template <typename T, bool MULTI>
__device__ __forceinline__ void tree_factor_body(DevSched s_p, TreeSched ts_p, DevNum<T> nm0_p, int B_p, int* ctr,
                                                 int* stall, long long limit, int fused, int u0, int nu, int tick,
                                                 const TreeJob<T>* jobs, const TreeSeg* segs, int nseg)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ TreeUnit su;                                    // the current unit and its front
    TreeFront& d = su.d;
    __shared__ int s_t, s_ok;
    __shared__ T s_rinv[64];                                   // reciprocal of every pivot (w <= 64)
    __shared__ __align__(16) unsigned char sj_raw[MULTI ? sizeof(TreeJob<T>) : 16];
    __shared__ int s_seg, s_job, s_switch;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    // units u0 .. u0 + nu - 1 of the chosen order (MULTI: nu tickets), tickets from counter ctr[tick]
    const int total = MULTI ? nu : nu * B_p;
    __shared__ int s_cut[kTreeMaxKids + 1];
    if (MULTI && tid == 0) s_job = -1;
    for (;;) {
        const int t = next_ticket(ctr + tick, ctr + 1, total, &s_t);
        if (t >= total) break;
        int ul, b;
        if (MULTI) {
            if (tid == 0) {                                        // segment of t (starts ascend)
                int lo = 0, hi = nseg - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (segs[mid].start <= t) lo = mid; else hi = mid - 1;
                }
                s_seg = lo;
                s_switch = segs[lo].job != s_job;
                if (s_switch) s_job = segs[lo].job;
            }
            __syncthreads();
            if (s_switch) {
                copy_words(reinterpret_cast<TreeJob<T>*>(sj_raw), jobs + s_job, 1, tid, 256);
                __syncthreads();
            }
            const TreeSeg sg = segs[s_seg];
            const int jb = reinterpret_cast<const TreeJob<T>*>(sj_raw)->B;
            ul = sg.ul0 + (t - sg.start) / jb;
            b = (t - sg.start) % jb;
        } else {
            ul = t / B_p;
            b = t - ul * B_p;
        }
        const TreeJob<T>* sj = reinterpret_cast<const TreeJob<T>*>(sj_raw);
        const DevSched& s = MULTI ? sj->s : s_p;
        const TreeSched& ts = MULTI ? sj->ts : ts_p;
        const DevNum<T>& nm0 = MULTI ? sj->nm : nm0_p;
        const int B = MULTI ? sj->B : B_p;
        int* done = (MULTI ? sj->ctr : ctr) + kCtrHead;
        int* fwd_done = done + (int64_t)B * ts.nq;                 // fused mode: forward-unit counters
        const TreeUnit* units = fused ? ts.unit_fused : ts.unit;
        T* M = reinterpret_cast<T*>(smraw);
        const int W = ts.map_w;
        const size_t off_map = align16(sizeof(T) * (size_t)ts.m_elems);
        int* smap = reinterpret_cast<int*>(smraw + off_map);       // child c: rows at 2cW, columns at (2c+1)W
        TreeKid* kids = reinterpret_cast<TreeKid*>(smraw + ts.kid_off);
        copy_words(&su, units + (MULTI ? 0 : u0) + ul, 1, tid, 256);
        __syncthreads();
        const FrontTile ut = su.u;
        const int q = ut.front;
        const DevNum<T> nm = nm0.at(b);
        if (ut.ti < 0) {                                           // forward-solve unit (fused mode)
            if (!fwd_unit<T, 256>(s, ts, nm, d, q, kids, s_cut, &s_ok, smraw, fwd_done + (int64_t)b * ts.nq,
                                  done + (int64_t)b * ts.nq, ctr + 1, limit)) {
                if (tid == 0) atomicExch(&nm.stat->timeout, 1);
                break;
            }
            __syncthreads();
            continue;
        }
        const int w = d.w, F = d.F, m = F - w, tsz = d.ts;
        const int i0 = ut.ti * tsz, j0 = ut.tj * tsz;
        const int nr = min(tsz, m - i0), nc = min(tsz, m - j0);
        const int Fr = w + nr, Fc = w + nc;
        const int nk = d.kid_end - d.kid_begin;
        const bool lead = ut.ti == 0 && ut.tj == 0;
        // ---- everything that does not depend on the children
        for (int e = tid; e < Fr * Fc; e += 256) M[e] = T(0);
        copy_words(kids, ts.kid + d.kid_begin, nk, tid, 256);
        for (int e = tid; e < nk * W; e += 256) {
            const int c = e / W, i = e - c * W;
            int vr = -1, vc = -1;
            if (i >= w) {
                const int* inv = ts.inv + d.inv_off + (int64_t)c * m;
                if (i - w < nr) vr = inv[i0 + i - w];
                if (i - w < nc) vc = inv[j0 + i - w];
            }
            smap[2 * c * W + i] = vr;
            smap[(2 * c + 1) * W + i] = vc;
        }
        __syncthreads();
        for (int64_t e = d.asm_begin + tid; e < d.asm_end; e += 256) {
            const int pos = s.asm_pos[e];
            const int bc = pos / F, a = pos - bc * F;
            const int lr = a < w ? a : ((unsigned)(a - w - i0) < (unsigned)nr ? a - i0 : -1);
            const int lc = bc < w ? bc : ((unsigned)(bc - w - j0) < (unsigned)nc ? bc - j0 : -1);
            if (lr >= 0 && lc >= 0) M[lr + lc * Fr] = nm.sv[s.asm_src[e]];
        }
        for (int c = ty; c < nk; c += 8) {                         // child rows t < k land on pivots
            const int k = kids[c].k;
            const int* rl = s.rel + kids[c].rel_ptr;
            for (int tt = tx; tt < k; tt += 32) {
                const int r = rl[tt];
                smap[2 * c * W + r] = tt;
                smap[(2 * c + 1) * W + r] = tt;
            }
        }
        // static-pivot floor (the scaling kernel's max |D K D|), loaded before the wait
        const T floorT = (T)(nm.pivot_eps * __longlong_as_double((long long)nm.stat->amax_bits));
        // ---- wait for the children (bounded; lane l of warp 0 polls children l, l + 32)
        if (tid == 0) {
            s_ok = 1;
            if (!MULTI && stall && t == 0 && *stall) {             // test hook: a wait nothing ends
                s_ok = bounded_wait(stall + 1, 1, ctr + 1, limit);
                *stall = 0;
            }
        }
        __syncthreads();
        if (s_ok && tid < 32) {
            const int ok = warp_wait_kids(done + (int64_t)b * ts.nq, kids, nk, false, ctr + 1, limit);
            if (tid == 0) s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) {
            if (tid == 0) atomicExch(&nm.stat->timeout, 1);
            break;
        }
        // ---- children's contributions, in child order for every entry; each
        // thread holds four entries of one row and keeps up to 16 loads in flight
        for (int i = tx; i < Fr; i += 32)
            for (int jb = ty; jb < Fc; jb += 32) {
                T acc[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[k] = jb + 8 * k < Fc ? M[i + (jb + 8 * k) * Fr] : T(0);
                for (int c = 0; c < nk; c += 4) {
                    T v[4][4];
                    unsigned valid = 0u;
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        const int cc = c + g;
                        const int sr = cc < nk ? smap[2 * cc * W + i] : -1;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int j = jb + 8 * k;
                            const int sc = (cc < nk && j < Fc) ? smap[(2 * cc + 1) * W + j] : -1;
                            const bool ok = sr >= 0 && sc >= 0;
                            v[g][k] = ok ? __ldcg(nm.cb + kids[cc].cb_off + sr + (int64_t)sc * kids[cc].mc) : T(0);
                            valid |= ok ? (1u << (4 * g + k)) : 0u;
                        }
                    }
#pragma unroll
                    for (int g = 0; g < 4; ++g)
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (valid & (1u << (4 * g + k))) acc[k] += v[g][k];
                }
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (jb + 8 * k < Fc) M[i + (jb + 8 * k) * Fr] = acc[k];
            }
        __syncthreads();
        // ---- w pivot steps of right-looking elimination without pivoting, one
        // reciprocal per pivot (l_ip = m_ip * (1 / u_pp))
        if (sizeof(T) == 4 && Fr <= 32 && Fc <= 32) {
            // single precision, blocked by 8 pivots (elim_step_f32), the
            // static-pivot events counted once
            int n_bad = 0, n_pert = 0;
            float* Mf = reinterpret_cast<float*>(M);
            const float fl = (float)floorT;
            for (int p0 = 0; p0 < w; p0 += 8) {
                const int pk = min(8, w - p0);
                if (pk == 8)
                    elim_step_f32<true>(Mf, Fr, Fc, p0, pk, fl, n_bad, n_pert);
                else
                    elim_step_f32<false>(Mf, Fr, Fc, p0, pk, fl, n_bad, n_pert);
            }
            if (ty == 0 && lead && (n_bad | n_pert)) {                 // warp-uniform
                if (tx == 0 && n_bad) atomicExch(&nm.stat->numeric_bad, 1);
                if (tx == 0 && n_pert) atomicAdd(&nm.stat->n_perturbed, n_pert);
            }
        } else if (Fr <= 32 && Fc <= 32) {
            // mini fronts of at most 32 x 32 (always when w <= 16). GB300 runs
            // one FP64 warp instruction per ~64 cycles per sub-partition, masked
            // lanes included, so the elimination is bound by the FP64
            // instructions issued. Warp 0 owns column p+1 only: at step p it
            // finishes the next pivot (lane 0), broadcasts its reciprocal and
            // stores column p+1 already scaled, so at step p+1 every other warp
            // reads l_i,p+1 and issues FMAs alone. Warps 1-7 own five adjacent
            // columns each from p+2 (lane -> row), a warp whose columns are all
            // eliminated issues nothing, and warp 4, which shares a
            // sub-partition with warp 0, takes the last group.
            if (ty == 0 && w > 0) {
                T r = T(0);
                if (tx == 0) {
                    const T pv = static_pivot(M[0], floorT, nm.stat, lead);
                    M[0] = pv;
                    r = pivot_rcp(pv);
                }
                r = __shfl_sync(0xffffffffu, r, 0);
                if (1 + tx < Fr) M[1 + tx] *= r;
            }
            __syncthreads();
            const int g = ty < 4 ? ty - 1 : (ty == 4 ? 6 : ty - 2);
            for (int p = 0; p < w; ++p) {
                const int i = p + 1 + tx;
                if (ty == 0) {
                    const int j = p + 1;
                    const bool act = i < Fr && j < Fc;
                    T mv = T(0);
                    if (act) {
                        const T l = M[i + p * Fr];
                        mv = M[i + j * Fr];
                        mv -= l * M[p + j * Fr];
                    }
                    if (p + 1 < w) {                               // warp-uniform
                        T r = T(0);
                        if (tx == 0) {
                            mv = static_pivot(mv, floorT, nm.stat, lead);
                            r = pivot_rcp(mv);
                        }
                        r = __shfl_sync(0xffffffffu, r, 0);
                        if (tx > 0) mv *= r;
                    }
                    if (act) M[i + j * Fr] = mv;
                } else {
                    const int jg = p + 2 + 5 * g;
                    if (jg < Fc && i < Fr) {
                        const T l = M[i + p * Fr];
                        T mv[5], uv[5];
#pragma unroll
                        for (int k = 0; k < 5; ++k) {
                            const int j = jg + k;
                            mv[k] = j < Fc ? M[i + j * Fr] : T(0);
                            uv[k] = j < Fc ? M[p + j * Fr] : T(0);
                        }
#pragma unroll
                        for (int k = 0; k < 5; ++k) mv[k] -= l * uv[k];
#pragma unroll
                        for (int k = 0; k < 5; ++k) {
                            const int j = jg + k;
                            if (j < Fc) M[i + j * Fr] = mv[k];
                        }
                    }
                }
                __syncthreads();
            }
        } else {
            if (tid == 0 && w > 0) {
                const T pv = static_pivot(M[0], floorT, nm.stat, lead);
                M[0] = pv;
                s_rinv[0] = pivot_rcp(pv);
            }
            __syncthreads();
            for (int p = 0; p < w; ++p) {
                const T rinv = s_rinv[p];
                if (p > 0 && ty == (p - 1) % 8)                    // deferred scaling of column p-1
                    for (int i = p + tx; i < Fr; i += 32) M[i + (p - 1) * Fr] *= s_rinv[p - 1];
                for (int i = p + 1 + tx; i < Fr; i += 32) {
                    const T l = M[i + p * Fr] * rinv;
                    for (int j = p + 1 + ty; j < Fc; j += 8) {
                        const T a = M[i + j * Fr] - l * M[p + j * Fr];
                        if (i == p + 1 && j == p + 1 && p + 1 < w) {
                            const T pv = static_pivot(a, floorT, nm.stat, lead);
                            M[i + j * Fr] = pv;
                            s_rinv[p + 1] = pivot_rcp(pv);
                        } else {
                            M[i + j * Fr] = a;
                        }
                    }
                }
                __syncthreads();
            }
            if (w > 0)
                for (int i = w + tid; i < Fr; i += 256) M[i + (w - 1) * Fr] *= s_rinv[w - 1];
            __syncthreads();
        }
        // ---- results: pivot block (lead unit), L21 rows (tj == 0), U12 columns (ti == 0), CB tile
        T* pan = nm.panel + d.panel_off;
        if (lead)
            for (int c = ty; c < w; c += 8)
                for (int a = tx; a < w; a += 32) pan[a + (int64_t)c * F] = M[a + c * Fr];
        if (ut.tj == 0)
            for (int c = ty; c < w; c += 8)
                for (int r = tx; r < nr; r += 32) pan[(w + i0 + r) + (int64_t)c * F] = M[(w + r) + c * Fr];
        if (ut.ti == 0) {
            T* U12 = pan + (int64_t)F * w;
            for (int c = ty; c < nc; c += 8)
                for (int a = tx; a < w; a += 32) U12[a + (int64_t)(j0 + c) * w] = M[a + (w + c) * Fr];
        }
        T* C = nm.cb + d.cb_off;
        for (int c = ty; c < nc; c += 8)
            for (int r = tx; r < nr; r += 32) C[(i0 + r) + (int64_t)(j0 + c) * m] = M[(w + r) + (w + c) * Fr];
        signal_done(done + (int64_t)b * ts.nq + q);
    }
}

// Entry points: in single precision the kernel is held to 64 registers, so
// that 4 CTAs fit on an SM; double precision keeps the compiler's choice.
template <typename T, bool MULTI>
__global__ void __launch_bounds__(256) tree_factor_kernel(DevSched s, TreeSched ts, DevNum<T> nm, int B, int* ctr,
                                                          int* stall, long long limit, int fused, int u0, int nu,
                                                          int tick, const TreeJob<T>* jobs, const TreeSeg* segs,
                                                          int nseg)
{
    tree_factor_body<T, MULTI>(s, ts, nm, B, ctr, stall, limit, fused, u0, nu, tick, jobs, segs, nseg);
}

template <bool MULTI>
__global__ void __launch_bounds__(256, 4) tree_factor_kernel_f32(DevSched s, TreeSched ts, DevNum<float> nm, int B,
                                                                 int* ctr, int* stall, long long limit, int fused,
                                                                 int u0, int nu, int tick, const TreeJob<float>* jobs,
                                                                 const TreeSeg* segs, int nseg)
{
    tree_factor_body<float, MULTI>(s, ts, nm, B, ctr, stall, limit, fused, u0, nu, tick, jobs, segs, nseg);
}

template <bool MULTI>
auto tree_factor_entry(const float*) { return tree_factor_kernel_f32<MULTI>; }
template <bool MULTI>
auto tree_factor_entry(const double*) { return tree_factor_kernel<double, MULTI>; }

// ------------------------------------------------------ forward substitution

// Pivot-block substitutions by one warp (w <= 32), lane i holding entry i in a
// register and the pivot entry broadcast with a shuffle: the same operations
// in the same order as the shared-memory loops of every other solve kernel.
// v (length >= w) and the blocks are in shared memory; called by warp 0.
// Forward, unit lower L (column-major, leading dimension ld): for p ascending,
// v_i -= l_ip v_p for i > p.
template <typename T>
__device__ __forceinline__ void warp_lower_solve(T* v, const T* L, int ld, int w)
{
    const int lane = threadIdx.x & 31;
    T x = lane < w ? v[lane] : T(0);
    T li[32];
#pragma unroll
    for (int p = 0; p < 32; ++p) li[p] = (p < w && lane < w) ? L[lane + p * ld] : T(0);
#pragma unroll
    for (int p = 0; p < 32; ++p) {
        if (p >= w) break;
        const T xp = __shfl_sync(0xffffffffu, x, p);
        if (lane > p && lane < w) x -= li[p] * xp;              // FP64 costs pipe time per active lane
    }
    if (lane < w) v[lane] = x;
    __syncwarp();
}

// Backward, upper U (column-major, leading dimension w) with reciprocals
// rcp_p = 1 / u_pp: for p descending, x_p = v_p * rcp_p, v_a -= u_ap x_p for a < p.
template <typename T>
__device__ __forceinline__ void warp_upper_solve(T* v, const T* U, const T* rcp, int w)
{
    const int lane = threadIdx.x & 31;
    T x = lane < w ? v[lane] : T(0);
    const T r = lane < w ? rcp[lane] : T(0);
    T ua[32];
#pragma unroll
    for (int p = 0; p < 32; ++p) ua[p] = (p < w && lane < w) ? U[lane + p * w] : T(0);
#pragma unroll
    for (int p = 31; p >= 0; --p) {
        if (p >= w) continue;
        if (lane == p) x *= r;                                   // one lane's multiply, not the warp's
        const T xp = __shfl_sync(0xffffffffu, x, p);
        if (lane < p) x -= ua[p] * xp;
    }
    if (lane < w) v[lane] = x;
    __syncwarp();
}

// Front q of instance b (128 threads): gather the pivot entries and the
// children's contribution vectors, solve with the unit lower pivot block,
// update the other rows with L21 and leave them as the contribution vector.
// Forward substitution of front q (already in d, its children in kids) by
// NT threads: gather the pivot entries and the children's contribution
// vectors, solve with the unit lower pivot block, update the other rows with
// L21 and leave them as the contribution vector. fac_done (fused mode): the
// front's own factorization units run in the same kernel; the unit then also
// waits for them and reads the panel through L2 after the wait.
// Returns false if a wait gave up (the caller stops).
template <typename T, int NT>
__device__ bool fwd_unit(const DevSched& s, const TreeSched& ts, const DevNum<T>& nm, const TreeFront& d, int q,
                         TreeKid* kids, int* s_cut, int* s_ok, unsigned char* smraw, int* done_b,
                         const int* fac_done, int* abort_flag, long long limit)
{
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31;
    T* v = reinterpret_cast<T*>(smraw);
    T* P = v + ts.max_F;                                        // staged panel (F x w) or L11 (w x w)
    T* sval = P + (ts.fwd_stage ? ts.max_fw : ts.max_w * ts.max_w);
    int* spos = reinterpret_cast<int*>(sval + kTreeStage);
    const int w = d.w, F = d.F, first = d.first;
    const int nk = d.kid_end - d.kid_begin;
    const T* pan = nm.panel + d.panel_off;
    const int ldp = ts.fwd_stage ? F : w;
    const bool fused = fac_done != nullptr;
    for (int a = tid; a < F; a += NT) v[a] = a < w ? nm.vec[first + a] : T(0);
    if (!fused) {
        if (ts.fwd_stage) {
            for (int c = tid >> 5; c < w; c += NW)
                for (int a = lane; a < F; a += 32) P[a + c * F] = pan[a + (int64_t)c * F];
        } else {
            for (int c = tid >> 5; c < w; c += NW)
                for (int a = lane; a < w; a += 32) P[a + c * w] = pan[a + (int64_t)c * F];
        }
    }
    copy_words(kids, ts.kid + d.kid_begin, nk, tid, NT);
    __syncthreads();
    if (tid == 0) {
        // children's entries, staged in passes of at most kTreeStage
        int acc = 0;
        s_cut[0] = 0;
        for (int c = 0; c < nk; ++c) {
            acc += kids[c].mc;
            s_cut[c + 1] = acc;
        }
    }
    __syncthreads();
    const bool one_pass = s_cut[nk] <= kTreeStage;
    if (one_pass)                                                 // positions do not depend on the children
        for (int c = 0; c < nk; ++c) {
            const int* rl = s.rel + kids[c].rel_ptr;
            for (int tt = tid; tt < kids[c].mc; tt += NT) spos[s_cut[c] + tt] = rl[tt];
        }
    if (tid < 32) {
        const int ok = warp_wait_kids(done_b, kids, nk, true, abort_flag, limit, fused ? fac_done + q : nullptr,
                                      d.units);
        if (tid == 0) *s_ok = ok;
    }
    __syncthreads();
    if (!*s_ok) return false;
    if (fused) {
        if (ts.fwd_stage) {
            for (int c = tid >> 5; c < w; c += NW)
                for (int a = lane; a < F; a += 32) P[a + c * F] = __ldcg(pan + a + (int64_t)c * F);
        } else {
            for (int c = tid >> 5; c < w; c += NW)
                for (int a = lane; a < w; a += 32) P[a + c * w] = __ldcg(pan + a + (int64_t)c * F);
        }
    }
    if (one_pass) {
        for (int c = 0; c < nk; ++c) {
            const T* cv = nm.cbv + kids[c].rel_ptr;
            for (int tt = tid; tt < kids[c].mc; tt += NT) sval[s_cut[c] + tt] = __ldcg(cv + tt);
        }
        __syncthreads();
        for (int c = 0; c < nk; ++c) {
            for (int tt = tid; tt < kids[c].mc; tt += NT) v[spos[s_cut[c] + tt]] += sval[s_cut[c] + tt];
            __syncthreads();
        }
    } else {
        __syncthreads();
        for (int c0 = 0; c0 < nk;) {
            int c1 = c0 + 1;                                      // at least one child per pass
            while (c1 < nk && s_cut[c1 + 1] - s_cut[c0] <= kTreeStage) ++c1;
            const int base = s_cut[c0];
            // stage (position, value) of children c0..c1-1 in one round of loads
            for (int c = c0; c < c1; ++c) {
                const int mc = kids[c].mc;
                const int* rl = s.rel + kids[c].rel_ptr;
                const T* cv = nm.cbv + kids[c].rel_ptr;
                const int off = s_cut[c] - base;
                if (off + mc <= kTreeStage) {
                    for (int tt = tid; tt < mc; tt += NT) {
                        spos[off + tt] = rl[tt];
                        sval[off + tt] = __ldcg(cv + tt);
                    }
                }
            }
            __syncthreads();
            for (int c = c0; c < c1; ++c) {
                const int mc = kids[c].mc;
                const int off = s_cut[c] - base;
                if (off + mc <= kTreeStage) {
                    for (int tt = tid; tt < mc; tt += NT) v[spos[off + tt]] += sval[off + tt];
                } else {                                          // a child larger than the stage
                    const int* rl = s.rel + kids[c].rel_ptr;
                    const T* cv = nm.cbv + kids[c].rel_ptr;
                    for (int tt = tid; tt < mc; tt += NT) v[rl[tt]] += __ldcg(cv + tt);
                }
                __syncthreads();
            }
            c0 = c1;
        }
    }
    if (tid < 32) {
        if (w <= 32)
            warp_lower_solve(v, P, ldp, w);
        else
            for (int p = 0; p < w; ++p) {
                const T xp = v[p];
                for (int i = p + 1 + lane; i < w; i += 32) v[i] -= P[i + p * ldp] * xp;
                __syncwarp();
            }
    }
    __syncthreads();
    for (int i = w + tid; i < F; i += NT) {
        T acc = v[i];
        if (ts.fwd_stage)
            for (int p = 0; p < w; ++p) acc -= P[i + p * F] * v[p];
        else if (fused)
            for (int p = 0; p < w; ++p) acc -= __ldcg(pan + i + (int64_t)p * F) * v[p];
        else
            for (int p = 0; p < w; ++p) acc -= pan[i + (int64_t)p * F] * v[p];
        v[i] = acc;
    }
    __syncthreads();
    for (int a = tid; a < w; a += NT) nm.vec[first + a] = v[a];
    T* cvo = nm.cbv + d.rel_ptr;
    for (int tt = tid; tt < F - w; tt += NT) cvo[tt] = v[w + tt];
    signal_done(done_b + q);
    return true;
}

// ------------------------------------------------------ backward substitution

// Asynchronous copy of one 4- or 8-byte word into shared memory (cp.async),
// and the wait for every copy this thread has issued.
__device__ __forceinline__ void cp_word(void* smem_dst, const void* gsrc, int bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Named barrier 1 over the first `nthr` threads counted from a warp boundary
// (the threads that stage a front; barrier 0 is __syncthreads).
__device__ __forceinline__ void bar_sync_staging(int nthr)
{
    asm volatile("bar.sync 1, %0;\n" ::"r"(nthr) : "memory");
}

// Forward substitution of the tree part by chains: the backward kernel's
// chains run bottom front first, chains in ascending order of their top
// front, so every chain that a bottom front waits on holds an earlier ticket.
// The bottom front of a chain waits for its children in the tree part (tops
// of earlier chains) and reads their contribution vectors from memory; every
// later front has the front before it as its only child in the tree part,
// whose contribution vector is still in shared memory, so it takes it from
// there through the relative indices, with no wait. Everything else a front
// reads (its own right-hand-side entries, its panel or pivot block, its
// children's relative indices and the contribution vectors of its children
// below the tree part) was written before the launch, so warps 1-3 copy the
// next front's share by cp.async while warp 0 solves with the current pivot
// block; descriptors come two fronts ahead, children's descriptors one ahead.
// Children are added in their stored order, one after another, and the L21
// update sums in pivot order: the results equal a front-by-front substitution
// bit for bit. Only the chain's top writes its contribution vector and
// signals completion.
template <typename T>
__global__ void __launch_bounds__(128) tree_fwd_kernel(DevSched s, TreeSched ts, DevNum<T> nm0, int B, int* ctr,
                                                       long long limit)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ TreeFront dd[3];
    __shared__ TreeKid kb[2][kTreeMaxKids];
    __shared__ int cut[2][kTreeMaxKids + 1];
    __shared__ int staged[2];
    __shared__ int s_t, s_ok;
    const int tid = threadIdx.x, lane = tid & 31;
    const int total = ts.nchains * B;
    int* done = ctr + kCtrHead;
    const int pw = ts.fwd_cstage ? ts.max_fw : ts.max_w * ts.max_w;    // panel F x w, or pivot block w x w
    const int ks = ts.fwd_kstage;                               // children's entries staged per front
    const int stage_len = ts.max_w + pw + ks;
    T* vb = reinterpret_cast<T*>(smraw);                        // v of the current and of the previous front
    T* stg = vb + 2 * ts.max_F;                                 // two staging buffers: y, P, children's values
    int* spos = reinterpret_cast<int*>(stg + 2 * stage_len);    // two buffers of children's relative indices
    // copies of front d's static share into buffer sb by threads t0 .. t0 +
    // nthr - 1 (whole warps); its children's descriptors are in kb[sb]
    auto stage = [&](int sb, const TreeFront& d, const DevNum<T>& nm, int t0, int nthr) {
        const int me = tid - t0, wi = me >> 5, nw = nthr >> 5;
        T* y = stg + sb * stage_len;
        T* P = y + ts.max_w;
        T* sv = P + pw;
        int* sp = spos + sb * ks;
        const int w = d.w, F = d.F, nk = d.kid_end - d.kid_begin;
        const T* pan = nm.panel + d.panel_off;
        for (int a = me; a < w; a += nthr) cp_word(y + a, nm.vec + d.first + a, (int)sizeof(T));
        if (ts.fwd_cstage) {
            for (int c = wi; c < w; c += nw)
                for (int a = lane; a < F; a += 32) cp_word(P + a + c * F, pan + a + (int64_t)c * F, (int)sizeof(T));
        } else {
            for (int c = wi; c < w; c += nw)
                for (int a = lane; a < w; a += 32) cp_word(P + a + c * w, pan + a + (int64_t)c * F, (int)sizeof(T));
        }
        if (wi == 0) {                                           // offsets: prefix sums of the children's orders
            int run = 0;
            for (int c0 = 0; c0 < nk; c0 += 32) {
                const int c = c0 + lane;
                int x = c < nk ? kb[sb][c].mc : 0;
                for (int o = 1; o < 32; o <<= 1) {
                    const int up = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += up;
                }
                if (c < nk) cut[sb][c + 1] = run + x;
                run += __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0) {
                cut[sb][0] = 0;
                staged[sb] = run <= ks ? 1 : 0;
            }
        }
        bar_sync_staging(nthr);
        if (staged[sb])
            for (int c = 0; c < nk; ++c) {
                const TreeKid& k = kb[sb][c];
                const int off = cut[sb][c];
                const int* rl = s.rel + k.rel_ptr;
                for (int tt = me; tt < k.mc; tt += nthr) {
                    cp_word(sp + off + tt, rl + tt, 4);
                    if (k.q < 0) cp_word(sv + off + tt, nm.cbv + k.rel_ptr + tt, (int)sizeof(T));
                }
            }
    };
    auto fetch_desc = [&](int slot, int q_) {
        constexpr int kWords = (int)(sizeof(TreeFront) / 4);
        static_assert(sizeof(TreeFront) % 4 == 0, "descriptor words");
        if (tid < kWords)
            cp_word(reinterpret_cast<int*>(&dd[slot]) + tid, reinterpret_cast<const int*>(ts.fr + q_) + tid, 4);
    };
    auto fetch_kids = [&](int sb, const TreeFront& d) {
        static_assert(sizeof(TreeKid) % 4 == 0, "descriptor words");
        const int words = (d.kid_end - d.kid_begin) * (int)(sizeof(TreeKid) / 4);
        const int* src = reinterpret_cast<const int*>(ts.kid + d.kid_begin);
        for (int e = tid; e < words; e += 128) cp_word(reinterpret_cast<int*>(kb[sb]) + e, src + e, 4);
    };
    for (;;) {
        const int t = next_ticket(ctr + 2, ctr + 1, total, &s_t);
        if (t >= total) break;
        const int cr = t / B, b = t - cr * B;
        const int ci = ts.nchains - 1 - cr;                     // ascending top front
        const int k0 = ts.bwd_chain_ptr[ci], k1 = ts.bwd_chain_ptr[ci + 1];
        const int len = k1 - k0;                                // position j: front bwd_chain[k1 - 1 - j]
        const DevNum<T> nm = nm0.at(b);
        fetch_desc(0, ts.bwd_chain[k1 - 1]);
        if (len > 1) fetch_desc(1, ts.bwd_chain[k1 - 2]);
        cp_wait_all();
        __syncthreads();
        fetch_kids(0, dd[0]);
        cp_wait_all();
        __syncthreads();
        stage(0, dd[0], nm, 0, 128);
        bool stop = false;
        int wprev = 0;
        // the bottom front waits for its children in the tree part while its
        // share is in flight
        if (tid < 32) {
            const int ok = warp_wait_kids(done + (int64_t)b * ts.nq, kb[0], dd[0].kid_end - dd[0].kid_begin, true,
                                          ctr + 1, limit);
            if (tid == 0) s_ok = ok;
        }
        for (int j = 0; j < len; ++j) {
            const int sb = j & 1, ds = j % 3;
            cp_wait_all();                                       // this front's share and descriptors
            __syncthreads();
            if (j == 0 && !s_ok) {
                if (tid == 0) atomicExch(&nm.stat->timeout, 1);
                stop = true;
                break;
            }
            const int w = dd[ds].w, F = dd[ds].F, first = dd[ds].first, nk = dd[ds].kid_end - dd[ds].kid_begin;
            if (j + 2 < len) fetch_desc((ds + 2) % 3, ts.bwd_chain[k1 - 3 - j]);
            if (j + 1 < len) fetch_kids(sb ^ 1, dd[(ds + 1) % 3]);
            T* v = vb + sb * ts.max_F;
            const T* pv = vb + (sb ^ 1) * ts.max_F;              // the previous front of the chain
            const T* y = stg + sb * stage_len;
            const T* P = y + ts.max_w;
            const T* sv = P + pw;
            const int* sp = spos + sb * ks;
            const bool st_ok = staged[sb] != 0;
            for (int a = tid; a < F; a += 128) v[a] = a < w ? y[a] : T(0);
            __syncthreads();
            for (int c = 0; c < nk; ++c) {
                const TreeKid& k = kb[sb][c];
                const int mc = k.mc;
                const int* rl = st_ok ? sp + cut[sb][c] : s.rel + k.rel_ptr;
                if (k.q < 0) {
                    if (st_ok)
                        for (int tt = tid; tt < mc; tt += 128) v[rl[tt]] += sv[cut[sb][c] + tt];
                    else
                        for (int tt = tid; tt < mc; tt += 128) v[rl[tt]] += __ldcg(nm.cbv + k.rel_ptr + tt);
                } else if (j > 0) {
                    for (int tt = tid; tt < mc; tt += 128) v[rl[tt]] += pv[wprev + tt];
                } else {
                    for (int tt = tid; tt < mc; tt += 128) v[rl[tt]] += __ldcg(nm.cbv + k.rel_ptr + tt);
                }
                __syncthreads();
            }
            cp_wait_all();                                       // the next front's children's descriptors
            __syncthreads();
            // warps 1-3 stage the next front while warp 0 solves this one
            if (j + 1 < len && tid >= 32) stage(sb ^ 1, dd[(ds + 1) % 3], nm, 32, 96);
            if (tid < 32) {
                const int ldp = ts.fwd_cstage ? F : w;
                if (w <= 32)
                    warp_lower_solve(v, P, ldp, w);
                else
                    for (int p = 0; p < w; ++p) {
                        const T xp = v[p];
                        for (int i = p + 1 + lane; i < w; i += 32) v[i] -= P[i + p * ldp] * xp;
                        __syncwarp();
                    }
            }
            __syncthreads();
            const T* pan = nm.panel + dd[ds].panel_off;
            for (int i = w + tid; i < F; i += 128) {
                T acc = v[i];
                if (ts.fwd_cstage)
                    for (int p = 0; p < w; ++p) acc -= P[i + p * F] * v[p];
                else
                    for (int p = 0; p < w; ++p) acc -= pan[i + (int64_t)p * F] * v[p];
                v[i] = acc;
            }
            __syncthreads();
            for (int a = tid; a < w; a += 128) nm.vec[first + a] = v[a];
            if (j == len - 1) {
                T* cvo = nm.cbv + dd[ds].rel_ptr;
                for (int tt = tid; tt < F - w; tt += 128) cvo[tt] = v[w + tt];
            }
            wprev = w;
        }
        if (stop) {
            cp_wait_all();                                       // no copy left in flight
            break;
        }
        signal_done(done + (int64_t)b * ts.nq + ts.bwd_chain[k0]);
        __syncthreads();
    }
}

// Chain c of instance b (TreeSched::bwd_chain), tickets in chain order
// (parents first): the solution entries of a front's other rows belong to its
// ancestors, which are complete once its parent is. The first front of a
// chain waits for its parent's chain and gathers those entries from the
// solution vector; every later front of the chain is the only tree child of
// the one before it, whose whole front (its pivots just solved and its other
// rows) is still in shared memory, so it takes them from there through its
// relative indices -- the same values, with no wait and no round trip
// through memory. The static data of the next front (pivot block, U12, own
// pivot entries, indices) is copied by cp.async into the second staging
// buffer while the current front is solved, and the descriptor of the front
// after it alongside (three descriptor slots). Completion is signalled once,
// for the last front of the chain: the only front whose children in the tree
// part are outside it.
template <typename T>
__global__ void __launch_bounds__(128) tree_bwd_kernel(DevSched s, TreeSched ts, DevNum<T> nm0, int B, int* ctr,
                                                       long long limit)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ TreeFront dd[3];
    __shared__ int s_t, s_ok;
    __shared__ T red[128];
    __shared__ T rcp[64];                                       // 1 / u_pp of the pivot block (w <= 64)
    const int tid = threadIdx.x, lane = tid & 31;
    const int total = ts.nchains * B;
    int* done = ctr + kCtrHead + ts.nq * B;                     // after the forward counters
    const int stage_len = ts.max_w + ts.max_w * ts.max_w + (ts.bwd_stage ? ts.max_wm : 0);
    T* vb = reinterpret_cast<T*>(smraw);                        // v of the two last fronts: vb, vb + max_F
    T* stg = vb + 2 * ts.max_F;                                 // staging buffers: y, Us, U12s (twice)
    int* rix = reinterpret_cast<int*>(stg + 2 * stage_len);     // index buffers (twice)
    // issue the copies of front d's static data into staging buffer sb, by
    // threads t0 .. t0 + nthr - 1 (whole warps) of the CTA
    auto stage = [&](int sb, const TreeFront& d, bool first_of_chain, const DevNum<T>& nm, int t0, int nthr) {
        const int me = tid - t0, wi = me >> 5, nw = nthr >> 5;
        T* y = stg + sb * stage_len;
        T* Us = y + ts.max_w;
        T* U12s = Us + ts.max_w * ts.max_w;
        int* ridx = rix + sb * ts.max_F;
        const int w = d.w, F = d.F, m = F - w;
        const T* pan = nm.panel + d.panel_off;
        const int* src = first_of_chain ? s.rows + d.rows_ptr + w : s.rel + d.rel_ptr;
        for (int tt = me; tt < m; tt += nthr) cp_word(ridx + tt, src + tt, 4);
        for (int a = me; a < w; a += nthr) cp_word(y + a, nm.vec + d.first + a, (int)sizeof(T));
        for (int c = wi; c < w; c += nw)
            for (int a = lane; a < w; a += 32) cp_word(Us + a + c * w, pan + a + (int64_t)c * F, (int)sizeof(T));
        if (ts.bwd_stage) {
            const T* U12 = pan + (int64_t)F * w;
            for (int e = me; e < w * m; e += nthr) cp_word(U12s + e, U12 + e, (int)sizeof(T));
        }
    };
    // descriptor of chain position k into slot k % 3, by cp.async
    auto fetch_desc = [&](int slot, int q_) {
        constexpr int kWords = (int)(sizeof(TreeFront) / 4);
        static_assert(sizeof(TreeFront) % 4 == 0, "descriptor words");
        if (tid < kWords)
            cp_word(reinterpret_cast<int*>(&dd[slot]) + tid, reinterpret_cast<const int*>(ts.fr + q_) + tid, 4);
    };
    for (;;) {
        const int t = next_ticket(ctr + 3, ctr + 1, total, &s_t);
        if (t >= total) break;
        const int ci = t / B, b = t - ci * B;
        const int k0 = ts.bwd_chain_ptr[ci], k1 = ts.bwd_chain_ptr[ci + 1];
        const DevNum<T> nm = nm0.at(b);
        fetch_desc(0, ts.bwd_chain[k0]);
        if (k0 + 1 < k1) fetch_desc(1, ts.bwd_chain[k0 + 1]);
        cp_wait_all();
        __syncthreads();
        stage(0, dd[0], true, nm, 0, 128);
        bool stop = false;
        int q = -1;
        for (int k = k0; k < k1; ++k) {
            const int sb = (k - k0) & 1, ds = (k - k0) % 3;
            q = ts.bwd_chain[k];
            cp_wait_all();                                       // this front's staging and the next descriptor
            if (k == k0 && tid < 32) {
                TreeKid par{};
                par.q = dd[ds].parent;
                const int ok = warp_wait_kids(done + (int64_t)b * ts.nq, &par, 1, true, ctr + 1, limit);
                if (tid == 0) s_ok = ok;
            }
            __syncthreads();
            if (k == k0 && !s_ok) {
                if (tid == 0) atomicExch(&nm.stat->timeout, 1);
                stop = true;
                break;
            }
            const int w = dd[ds].w, F = dd[ds].F, first = dd[ds].first, m = F - w;
            const T* U12 = nm.panel + dd[ds].panel_off + (int64_t)F * w;
            const T* y = stg + sb * stage_len;
            const T* Us = y + ts.max_w;
            const T* U12s = Us + ts.max_w * ts.max_w;
            const int* ridx = rix + sb * ts.max_F;
            T* v = vb + sb * ts.max_F;
            const T* pv = vb + (sb ^ 1) * ts.max_F;              // the previous front of the chain
            if (k + 2 < k1) fetch_desc((ds + 2) % 3, ts.bwd_chain[k + 2]);
            for (int a = tid; a < w; a += 128) rcp[a] = pivot_rcp(Us[a + a * w]);
            if (k == k0)
                for (int tt = tid; tt < m; tt += 128) v[w + tt] = __ldcg(nm.vec + ridx[tt]);
            else
                for (int tt = tid; tt < m; tt += 128) v[w + tt] = pv[ridx[tt]];
            __syncthreads();
            // y_a - sum_t U12[a, t] x_t, in the order every backward kernel uses:
            // in sequence for m <= kSeqSum, else 128 / w interleaved partial sums per row
            if (m <= kSeqSum) {
                for (int a = tid; a < w; a += 128) {
                    T acc = y[a];
                    if (ts.bwd_stage)
                        for (int tt = 0; tt < m; ++tt) acc -= U12s[a + tt * w] * v[w + tt];
                    else
                        for (int tt = 0; tt < m; ++tt) acc -= U12[a + (int64_t)tt * w] * v[w + tt];
                    v[a] = acc;
                }
            } else {
                const int G = 128 / w;
                T part = T(0);
                if (tid < G * w) {
                    // in sequence, four terms' loads issued ahead of their FMAs
                    const int a = tid % w, g = tid / w;
                    const T* Ua = ts.bwd_stage ? U12s + a : U12 + a;
                    int tt = g;
                    for (; tt + 3 * G < m; tt += 4 * G) {
                        T u[4], x[4];
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            u[r] = Ua[(int64_t)(tt + r * G) * w];
                            x[r] = v[w + tt + r * G];
                        }
#pragma unroll
                        for (int r = 0; r < 4; ++r) part += u[r] * x[r];
                    }
                    for (; tt < m; tt += G) part += Ua[(int64_t)tt * w] * v[w + tt];
                }
                red[tid] = part;
                __syncthreads();
                for (int a = tid; a < w; a += 128) {
                    T acc = T(0);
                    for (int g = 0; g < G; ++g) acc += red[a + g * w];
                    v[a] = y[a] - acc;
                }
            }
            __syncthreads();
            // warps 1-3 stage the next front while warp 0 solves this one
            if (k + 1 < k1 && tid >= 32) stage(sb ^ 1, dd[(ds + 1) % 3], false, nm, 32, 96);
            if (tid < 32) {
                if (w <= 32)
                    warp_upper_solve(v, Us, rcp, w);
                else
                    for (int p = w - 1; p >= 0; --p) {
                        const T xp = v[p] * rcp[p];
                        __syncwarp();
                        if (lane == 0) v[p] = xp;
                        for (int a = lane; a < p; a += 32) v[a] -= Us[a + p * w] * xp;
                        __syncwarp();
                    }
            }
            __syncthreads();
            for (int a = tid; a < w; a += 128) nm.vec[first + a] = v[a];
        }
        if (stop) break;
        signal_done(done + (int64_t)b * ts.nq + q);
        __syncthreads();
    }
}

}  // namespace

template <typename T>
cudaError_t tree_grid(int kind, size_t smem, int* grid)
{
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
    if (kind == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tree_factor_entry<false>((const T*)nullptr), 256, smem);
    else if (kind == 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tree_factor_entry<true>((const T*)nullptr), 256, smem);
    else if (kind == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tree_fwd_kernel<T>, 128, smem);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tree_bwd_kernel<T>, 128, smem);
    if (e != cudaSuccess) return e;
    // at most kTreeCtasPerSm resident CTAs per SM by default (measured: more
    // share an SM's FP64 pipe without hiding more of the dependency waits);
    // KKT_TREE_CTAS_PER_SM overrides the cap (a tuning knob)
    int cap = kTreeCtasPerSm;
    if (const char* env = std::getenv("KKT_TREE_CTAS_PER_SM")) {
        const int c = std::atoi(env);
        if (c > 0) cap = c;
    }
    per = std::min(per, cap);
    *grid = sms * (per > 0 ? per : 1);
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_tree_factor(const DevSched& s, const TreeSched& t, const DevNum<T>& nm, int batch, int* ctr,
                               int* stall, long long spin_limit, int grid, size_t smem, int fused, int u0, int nu,
                               int tick, cudaStream_t st)
{
    const int g = std::min<long long>(grid, (long long)nu * batch);
    if (g <= 0) return cudaSuccess;
    if ((fused ? t.unit_fused : t.unit) == nullptr || t.fr == nullptr || t.kid == nullptr)
        return cudaErrorInvalidValue;                         // schedule not uploaded: never launch on it
    if (u0 < 0 || nu < 0 || u0 + nu > (fused ? t.nunits_fused : t.nunits) || (tick != 0 && tick != 3))
        return cudaErrorInvalidValue;
    tree_factor_entry<false>((const T*)nullptr)<<<g, 256, smem, st>>>(s, t, nm, batch, ctr, stall, spin_limit, fused, u0, nu, tick,
                                                       nullptr, nullptr, 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tree_factor_group(const TreeJob<T>* jobs, const TreeSeg* segs, int nseg, int total, int* gctr,
                                     long long spin_limit, int grid, size_t smem, cudaStream_t st)
{
    const int g = std::min(grid, total);
    if (g <= 0) return cudaSuccess;
    if (!jobs || !segs || nseg <= 0 || !gctr) return cudaErrorInvalidValue;
    tree_factor_entry<true>((const T*)nullptr)<<<g, 256, smem, st>>>(DevSched{}, TreeSched{}, DevNum<T>{}, 1, gctr, nullptr,
                                                      spin_limit, 0, 0, total, 0, jobs, segs, nseg);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tree_fwd(const DevSched& s, const TreeSched& t, const DevNum<T>& nm, int batch, int* ctr,
                            long long spin_limit, int grid, size_t smem, cudaStream_t st)
{
    const int g = std::min<long long>(grid, (long long)t.nq * batch);
    if (g <= 0) return cudaSuccess;
    if (t.fr == nullptr || t.kid == nullptr) return cudaErrorInvalidValue;
    tree_fwd_kernel<T><<<g, 128, smem, st>>>(s, t, nm, batch, ctr, spin_limit);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tree_bwd(const DevSched& s, const TreeSched& t, const DevNum<T>& nm, int batch, int* ctr,
                            long long spin_limit, int grid, size_t smem, cudaStream_t st)
{
    const int g = std::min<long long>(grid, (long long)t.nchains * batch);
    if (g <= 0) return cudaSuccess;
    if (t.fr == nullptr || t.bwd_chain == nullptr || t.bwd_chain_ptr == nullptr) return cudaErrorInvalidValue;
    tree_bwd_kernel<T><<<g, 128, smem, st>>>(s, t, nm, batch, ctr, spin_limit);
    return cudaGetLastError();
}

#define KKT_TREE_INST(T)                                                                                          \
    template cudaError_t tree_grid<T>(int, size_t, int*);                                                          \
    template cudaError_t launch_tree_factor<T>(const DevSched&, const TreeSched&, const DevNum<T>&, int, int*,     \
                                               int*, long long, int, size_t, int, int, int, int, cudaStream_t);    \
    template cudaError_t launch_tree_fwd<T>(const DevSched&, const TreeSched&, const DevNum<T>&, int, int*,        \
                                            long long, int, size_t, cudaStream_t);                                 \
    template cudaError_t launch_tree_bwd<T>(const DevSched&, const TreeSched&, const DevNum<T>&, int, int*,        \
                                            long long, int, size_t, cudaStream_t);                                 \
    template cudaError_t launch_tree_factor_group<T>(const TreeJob<T>*, const TreeSeg*, int, int, int*, long long, \
                                                     int, size_t, cudaStream_t);
KKT_TREE_INST(double)
KKT_TREE_INST(float)

template <typename K>
static cudaError_t allow_smem_tree(K kernel, int optin)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

cudaError_t configure_tree_kernels(int optin)
{
    cudaError_t e;
    if ((e = allow_smem_tree(tree_factor_entry<false>((const double*)nullptr), optin))) return e;
    if ((e = allow_smem_tree(tree_factor_entry<false>((const float*)nullptr), optin))) return e;
    if ((e = allow_smem_tree(tree_factor_entry<true>((const double*)nullptr), optin))) return e;
    if ((e = allow_smem_tree(tree_factor_entry<true>((const float*)nullptr), optin))) return e;
    if ((e = allow_smem_tree(tree_fwd_kernel<double>, optin))) return e;
    if ((e = allow_smem_tree(tree_fwd_kernel<float>, optin))) return e;
    if ((e = allow_smem_tree(tree_bwd_kernel<double>, optin))) return e;
    if ((e = allow_smem_tree(tree_bwd_kernel<float>, optin))) return e;
    return cudaSuccess;
}

}  // namespace kktgb
