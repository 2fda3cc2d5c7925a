// CUDA kernels of the KKT refactor / solve / refine path (sm_103a).
//
// Numeric factorization is multifrontal over the supernodal assembly tree
// (one launch group per tree level): every front is a dense F x F matrix
// assembled from the scaled entries of K and its children's contribution
// blocks, whose first w columns/rows are factored without pivoting (static
// perturbation of tiny pivots), leaving the Schur complement as the front's
// contribution block. This computes the same L and U as the left-looking
// column LU of P (D K D) P^T in the paper's Alg. 1 refactor step, only with
// the updates grouped by subtree.
#include "kernels.cuh"

#include <math.h>

namespace kktgb {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Exact power-of-two arithmetic on IEEE bit patterns (integer pipes only; the
// FP64 pipe of this GPU issues one warp instruction per ~64 cycles in each
// sub-partition).
// scale2(x, e) = x * 2^e for a non-negative finite x; exact. Zero stays zero;
// results that would leave the normal range, and subnormal inputs, take the
// multiply.
__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a > b ? a : b; }
__device__ __forceinline__ unsigned long long warp_umax(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) v = umax64(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ int exp_of_pow2(double d)               // d = 2^k exactly
{
    return (int)((__double_as_longlong(d) >> 52) & 0x7ff) - 1023;
}
__device__ __forceinline__ unsigned long long scale2_bits(unsigned long long xb, int e)
{
    if (xb == 0ull) return 0ull;
    const int E = (int)(xb >> 52);                                 // biased exponent (sign bit is clear)
    const int En = E + e;
    if (E >= 1 && E <= 2046 && En >= 1 && En <= 2046) return xb + ((unsigned long long)(long long)e << 52);
    return (unsigned long long)__double_as_longlong(__longlong_as_double((long long)xb) * ldexp(1.0, e));
}

// 2^round(-log2(r)/2) with halves rounded up, r > 0, decided on the binary
// exponent only: r = m 2^e, m in [1/2, 1).
//   m == 1/2  : log2 r = e - 1 exactly         -> floor((2 - e) / 2)
//   otherwise : log2 r in (e - 1, e)            -> (1 - e)/2 for odd e, -e/2 for even e
__device__ __forceinline__ double pow2_inv_sqrt(double r)
{
    int e;
    double m = frexp(r, &e);
    int k;
    if (m == 0.5) {
        int t = 2 - e;
        k = t >= 0 ? t / 2 : -((1 - t) / 2);
    } else if (e & 1) {
        k = (1 - e) / 2;
    } else {
        k = -(e / 2);
    }
    return ldexp(1.0, k);
}

// Exponent k of pow2_inv_sqrt(r) from the bits of a positive normal r:
// r = (0.5 + M / 2^53) * 2^(E - 1022).
// The same decision for a positive normal number given by its biased
// exponent E and whether it is an exact power of two (m == 1/2).
__device__ __forceinline__ int pow2_inv_sqrt_exp_of(int E, bool pow2)
{
    const int e = E - 1022;
    if (pow2) {
        const int t = 2 - e;
        return t >= 0 ? t / 2 : -((1 - t) / 2);
    }
    return (e & 1) ? (1 - e) / 2 : -(e / 2);
}

__device__ __forceinline__ int pow2_inv_sqrt_exp(unsigned long long rb)
{
    const int E = (int)(rb >> 52);
    if (E == 0) return exp_of_pow2(pow2_inv_sqrt(__longlong_as_double((long long)rb)));   // subnormal
    return pow2_inv_sqrt_exp_of(E, (rb & 0x000fffffffffffffull) == 0ull);
}

// ------------------------------------------------------------------ Ruiz

// ---------------------------------------------------------- equilibration

// Every pass over K runs on its sliced copy (SellPlan): a warp per slice of 32
// rows, a lane per row, the row's entries k = 0, 1, ... at slots
// off + 32 k + lane (coalesced across the warp). Row maxima and row sums are
// then formed by one lane in sequence, with no cross-lane reduction: on this
// GPU an FP64 warp instruction costs the FP64 pipe the same whether 32 lanes or
// one do useful work, so the eight-lanes-per-row layout with shuffle sums spent
// most of its FP64 issue on the reductions.
constexpr int kSellWarps = 8;                      // slices per 256-thread block
constexpr unsigned kKeySpecial = 0xffffu;          // subnormal, infinite or NaN entry

// Exponent key of |k|: 0 for zero, (E << 1) | (mantissa != 0) for a normal
// number of biased exponent E, kKeySpecial otherwise.
__device__ __forceinline__ unsigned exp_key(double k)
{
    const unsigned long long b = abs_bits(k);
    if (b == 0ull) return 0u;
    const unsigned E = (unsigned)(b >> 52);
    if (E == 0u || E == 2047u) return kKeySpecial;
    return (E << 1) | ((b & 0x000fffffffffffffull) != 0ull ? 1u : 0u);
}

// Slots a lane loads ahead in the sliced kernels: its next kSellChunk keys
// (or values) and column indices are loaded first, then the kSellChunk
// gathers, then the arithmetic, so that every lane keeps that many independent
// loads in flight instead of walking one key -> column -> gather chain at a time.
constexpr int kSellChunk = 8;

// One Ruiz iteration, r_i = max_j |d_i k_ij d_j|, d_i <- d_i 2^round(-log2(r_i)/2),
// integer-only: every d is a power of two, so |d_i k_ij d_j| is |k_ij| with
// its exponent raised by e_i + e_j. Iteration 0 first copies K from the
// caller's CSR values into the sliced copy and writes the keys (load_only:
// nothing else, d = 1). Later iterations read the 2-byte keys and the column
// indices only: the row maximum has the largest shifted exponent, and a
// nonzero mantissa at that exponent is all pow2_inv_sqrt's rounding needs to
// know (the maximum is an exact power of two only if every entry at the top
// exponent is). A row with a special key, or a shifted exponent outside the
// normal range, is redone on the values (scale2_bits on the copy), the
// arithmetic of the by-value definition. Iteration 0 starts from d = 1 without
// reading din and writes 1 to din as well as the new d to dout. An iteration
// that changes no d_i leaves dout equal to din, bit for bit, so both buffers
// already hold the fixed point and every later iteration returns at once.
__global__ void __launch_bounds__(256) ruiz_sell_kernel(DevSched s, const double* __restrict__ v, int64_t bs_nnz,
                                                        double* kcopy, unsigned short* keys, int64_t bs_slot,
                                                        double* din, double* __restrict__ dout, DevStat* stat,
                                                        int it, int load_only)
{
    const int inst = blockIdx.y;
    if (it > 0 && stat[inst].ruiz_changed[it - 1] == 0) return;   // uniform over the grid
    v += (int64_t)inst * bs_nnz;
    kcopy += (int64_t)inst * bs_slot;
    keys += (int64_t)inst * bs_slot;
    din += (int64_t)inst * s.n;
    dout += (int64_t)inst * s.n;
    const int lane = threadIdx.x & 31;
    const int slice = blockIdx.x * kSellWarps + (threadIdx.x >> 5);
    int changed = 0;
    if (slice < s.nslices) {
        const int row = s.sell_row[slice * 32 + lane];
        const int64_t o0 = s.sell_off[slice] + lane, o1 = s.sell_off[slice + 1];
        const int ei = (row >= 0 && it > 0) ? exp_of_pow2(din[row]) : 0;
        unsigned m = 0u;
        bool special = false;
        if (it == 0) {
            for (int64_t ob = o0; ob < o1; ob += 32 * kSellChunk) {
                int src[kSellChunk];
#pragma unroll
                for (int u = 0; u < kSellChunk; ++u) {
                    const int64_t o = ob + 32 * u;
                    src[u] = o < o1 ? s.sell_src[o] : -1;
                }
                double k[kSellChunk];
#pragma unroll
                for (int u = 0; u < kSellChunk; ++u) k[u] = src[u] >= 0 ? v[src[u]] : 0.0;
#pragma unroll
                for (int u = 0; u < kSellChunk; ++u) {
                    const int64_t o = ob + 32 * u;
                    if (o < o1) {
                        const unsigned key = exp_key(k[u]);
                        kcopy[o] = k[u];
                        keys[o] = (unsigned short)key;
                        if (key == kKeySpecial) special = true;
                        else m = key > m ? key : m;
                    }
                }
            }
        } else {
            for (int64_t ob = o0; ob < o1; ob += 32 * kSellChunk) {
                unsigned key[kSellChunk];
                int c[kSellChunk];
#pragma unroll
                for (int u = 0; u < kSellChunk; ++u) {
                    const int64_t o = ob + 32 * u;
                    key[u] = o < o1 ? keys[o] : 0u;
                    c[u] = o < o1 ? s.sell_ci[o] : -1;
                }
                int ej[kSellChunk];
#pragma unroll
                for (int u = 0; u < kSellChunk; ++u)
                    ej[u] = (key[u] != 0u && key[u] != kKeySpecial) ? exp_of_pow2(din[c[u]]) : 0;
#pragma unroll
                for (int u = 0; u < kSellChunk; ++u) {
                    if (key[u] == 0u) continue;
                    if (key[u] == kKeySpecial) { special = true; continue; }
                    const int E = (int)(key[u] >> 1) + ei + ej[u];
                    if (E < 1 || E > 2046) { special = true; continue; }
                    const unsigned sk = ((unsigned)E << 1) | (key[u] & 1u);
                    m = sk > m ? sk : m;
                }
            }
        }
        if (row >= 0 && !load_only) {
            int e = 0;
            if (special) {
                unsigned long long mk = 0ull;
                for (int64_t o = o0; o < o1; o += 32) {
                    const int c = s.sell_ci[o];
                    if (c < 0) continue;
                    const int ej = it > 0 ? exp_of_pow2(din[c]) : 0;
                    const unsigned long long a = scale2_bits(abs_bits(kcopy[o]), ei + ej);
                    mk = a > mk ? a : mk;
                }
                e = mk ? pow2_inv_sqrt_exp(mk) : 0;
            } else if (m) {
                e = pow2_inv_sqrt_exp_of((int)(m >> 1), (m & 1u) == 0u);
            }
            const unsigned long long dib = (unsigned long long)(ei + 1023) << 52;   // d_i (1 in iteration 0)
            dout[row] = __longlong_as_double((long long)scale2_bits(dib, e));
            if (it == 0) din[row] = 1.0;
            changed = e != 0;
        } else if (row >= 0) {
            dout[row] = 1.0;
            din[row] = 1.0;
        }
    }
    // one flag write per block (a write per row would serialise on one address)
    if (__syncthreads_or(changed) && threadIdx.x == 0) stat[inst].ruiz_changed[it] = 1;
}

// D K D in factor precision (sliced layout: the assembly reads it through
// asm_src), max |D K D| (static-pivot reference) and ||K||_inf, whose row sums
// each lane forms in CSR order.
template <typename T>
__global__ void __launch_bounds__(256) scale_sell_kernel(DevSched s, DevNum<T> nm0)
{
    const DevNum<T> nm = nm0.at(blockIdx.y);
    const double* __restrict__ d = nm.d;
    const int lane = threadIdx.x & 31;
    const int slice = blockIdx.x * kSellWarps + (threadIdx.x >> 5);
    unsigned long long amb = 0ull, rsb = 0ull;
    if (slice < s.nslices) {
        const int row = s.sell_row[slice * 32 + lane];
        const int64_t o0 = s.sell_off[slice] + lane, o1 = s.sell_off[slice + 1];
        const int ei = row >= 0 ? exp_of_pow2(d[row]) : 0;
        double rsum = 0.0;
        for (int64_t ob = o0; ob < o1; ob += 32 * kSellChunk) {
            double k[kSellChunk];
            int c[kSellChunk];
#pragma unroll
            for (int u = 0; u < kSellChunk; ++u) {
                const int64_t o = ob + 32 * u;
                c[u] = o < o1 ? s.sell_ci[o] : -1;
                k[u] = o < o1 ? nm.kcopy[o] : 0.0;
            }
            int ej[kSellChunk];
#pragma unroll
            for (int u = 0; u < kSellChunk; ++u) ej[u] = c[u] >= 0 ? exp_of_pow2(d[c[u]]) : 0;
#pragma unroll
            for (int u = 0; u < kSellChunk; ++u) {
                const int64_t o = ob + 32 * u;
                if (o < o1) {
                    T out = T(0);
                    if (c[u] >= 0) {
                        const unsigned long long ab = scale2_bits(abs_bits(k[u]), ei + ej[u]);
                        const unsigned long long sb =
                            ab | ((unsigned long long)__double_as_longlong(k[u]) & 0x8000000000000000ull);
                        out = (T)__longlong_as_double((long long)sb);     // d_i k d_j, exact
                        amb = ab > amb ? ab : amb;
                        rsum += fabs(k[u]);
                    }
                    nm.sv[o] = out;
                }
            }
        }
        rsb = abs_bits(rsum);
    }
    // maxima of non-negative doubles as maxima of their bit patterns (integer shuffles)
    amb = warp_umax(amb);
    rsb = warp_umax(rsb);
    __shared__ unsigned long long s_am[kSellWarps], s_rs[kSellWarps];
    const int wid = threadIdx.x >> 5;
    if (lane == 0) { s_am[wid] = amb; s_rs[wid] = rsb; }
    __syncthreads();
    // one atomic per block and quantity (per-row atomics serialise on one address)
    if (threadIdx.x == 0) {
        unsigned long long a = 0ull, r = 0ull;
        for (int q = 0; q < kSellWarps; ++q) { a = umax64(a, s_am[q]); r = umax64(r, s_rs[q]); }
        atomicMax(&nm.stat->amax_bits, a);
        atomicMax(&nm.stat->knorm_bits, r);
    }
}

// sum_k kv[o_k] x[c_k] over the slots of one lane's row, in slot (= CSR) order
__device__ __forceinline__ double sell_row_dot(const DevSched& s, const double* __restrict__ kv,
                                               const double* __restrict__ x, int64_t o0, int64_t o1)
{
    double acc = 0.0;
    for (int64_t ob = o0; ob < o1; ob += 32 * kSellChunk) {
        double k[kSellChunk];
        int c[kSellChunk];
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u) {
            const int64_t o = ob + 32 * u;
            c[u] = o < o1 ? s.sell_ci[o] : -1;
            k[u] = o < o1 ? kv[o] : 0.0;
        }
        double xv[kSellChunk];
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u) xv[u] = c[u] >= 0 ? x[c[u]] : 0.0;
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u)
            if (c[u] >= 0) acc = fma(k[u], xv[u], acc);
    }
    return acc;
}

// ---------------------------------------------------------- front kernels

// The pivot of one elimination step, computed by every calling thread from
// the same entry x (no divergent branch, no shared-memory broadcast): the
// static pivot and its reciprocal (pivot_rcp's value: the Newton step, the
// division outside its range). The static-pivot events are accumulated in
// bad / pert and counted once per front by the caller. Single precision
// only: measured on GB300, FP64 instructions cost pipe time per active lane,
// so in double precision one lane computes the pivot and shares it.
template <typename T>
__device__ __forceinline__ T uniform_pivot(T x, T floorT, T& r, bool& bad, int& pert)
{
    bool b1, p1;
    const T pv = static_pivot_sel(x, floorT, b1, p1);
    r = pivot_rcp_fast(pv);
    if (!pivot_rcp_fast_ok(pv)) r = T(1) / pv;
    bad |= b1;
    pert += (int)p1;
    return pv;
}

__device__ __forceinline__ void count_pivot_events(DevStat* stat, bool bad, int pert)
{
    if (bad) atomicExch(&stat->numeric_bad, 1);
    if (pert) atomicAdd(&stat->n_perturbed, pert);
}

// Original entries of front f into the full F x F front Fm (shared memory):
// NT threads, four independent gathers in flight per thread.
template <typename T, int NT>
__device__ __forceinline__ void assemble_original(const DevSched& s, const DevNum<T>& nm, int f, int tid, T* Fm)
{
    const int64_t e0 = s.asm_ptr[f], e1 = s.asm_ptr[f + 1];
    for (int64_t e = e0 + tid; e < e1; e += NT * 4) {
        int pos[4];
        T val[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t ee = e + NT * u;
            pos[u] = ee < e1 ? s.asm_pos[ee] : -1;
            val[u] = ee < e1 ? nm.sv[s.asm_src[ee]] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (pos[u] >= 0) Fm[pos[u]] = val[u];
    }
}

// Loops over the entries of dense blocks use fixed two-dimensional thread
// layouts (rows across lanes, columns across lane groups or warps), so no
// thread divides by a run-time extent inside a loop: an integer division
// costs tens of instructions, more than the arithmetic it would index (the
// child-block adds of the warp kernel divide once per child and then step).

// Fronts with F <= 32: one warp per front, the whole front in shared memory.
// Lanes form an 8 x 4 grid over (row, column) of every block loop.
constexpr int kWarpCbBatch = 8;        // contribution-block loads in flight per lane

__device__ __forceinline__ void cp_async_word(void* smem_dst, const void* gsrc, int bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Contribution block of one child (mc x mc, column-major, contiguous at cb)
// into the front Fm (leading dimension F) at the child's relative indices:
// Fm[rel[a] + rel[b] F] += cb[a + b mc]. The values come from vals (global
// or shared), the indices from rl held by lanes 0..mc-1; every lane takes
// entries e = lane + 32 t, kWarpCbBatch loads issued before any update.
template <typename T>
__device__ __forceinline__ void warp_add_child(const T* vals, int mc, int rl, int F, int lane, T* Fm)
{
    const int ne = mc * mc, q = 32 / mc, r = 32 - q * mc;
    int a = lane % mc, b = lane / mc;                                 // entry lane = a + b mc
    if (__isShared(vals)) {                                           // staged: no loads to batch
        for (int e = lane; e - lane < ne; e += 32) {                  // warp-uniform trip count
            const int ra = __shfl_sync(kFull, rl, a), rb = __shfl_sync(kFull, rl, b);
            if (e < ne) Fm[ra + rb * F] += vals[e];
            a += r;
            b += q;
            if (a >= mc) { a -= mc; ++b; }
        }
        return;
    }
    for (int e0 = 0; e0 < ne; e0 += 32 * kWarpCbBatch) {
        T val[kWarpCbBatch];
        int pos[kWarpCbBatch];
#pragma unroll
        for (int t = 0; t < kWarpCbBatch; ++t) {
            const int e = e0 + lane + 32 * t;
            val[t] = e < ne ? vals[e] : T(0);
            pos[t] = e < ne ? -1 : -2;
        }
#pragma unroll
        for (int t = 0; t < kWarpCbBatch; ++t) {
            const int ra = __shfl_sync(kFull, rl, a), rb = __shfl_sync(kFull, rl, b);
            if (pos[t] == -1) pos[t] = ra + rb * F;
            a += r;
            b += q;
            if (a >= mc) { a -= mc; ++b; }
        }
#pragma unroll
        for (int t = 0; t < kWarpCbBatch; ++t)
            if (pos[t] >= 0) Fm[pos[t]] += val[t];
    }
}

// Forward step of front f with its factored front Fm (leading dimension F)
// still in shared memory, nl lanes (lane l of them; sync: their mask): v holds
// the pivot rows of the step vector plus the children's vectors. The
// operations, in order, of solve_fwd_kernel: the unit lower solve with L11,
// then each contribution row's sum over the pivots in sequence; the pivot
// rows go back to the step vector and the contribution rows to the front's
// vector for its parent.
template <typename T>
__device__ __forceinline__ void front_forward(const DevSched& s, const DevNum<T>& nm, int f, int first, int w, int F,
                                              const T* Fm, T* v, int l, int nl, unsigned mask)
{
    for (int p = 0; p < w; ++p) {
        const T xp = v[p];
        for (int i = p + 1 + l; i < w; i += nl) v[i] -= Fm[i + p * F] * xp;
        __syncwarp(mask);
    }
    for (int i = w + l; i < F; i += nl) {
        T acc = v[i];
        for (int p = 0; p < w; ++p) acc -= Fm[i + p * F] * v[p];
        v[i] = acc;
    }
    __syncwarp(mask);
    for (int a = l; a < w; a += nl) nm.vec[first + a] = v[a];
    T* cv = nm.cbv + s.rel_ptr[f];
    for (int t = l; t < F - w; t += nl) cv[t] = v[w + t];
}

// The children of front f added to Fm in child order, one warp. Lane k holds
// the descriptor of child k (32 at a time). Consecutive children whose
// blocks fit the warp's staging area (stage_v values, stage_r relative
// indices) are copied there by cp.async, all copies in flight together, so
// a front with many children waits for memory about once instead of once per
// child; a child too large for the staging area is read from global memory.
// With v (fused forward step) every child's vector is added to v as well,
// staged in scv beside its relative indices.
template <typename T>
__device__ __forceinline__ void warp_children(const DevSched& s, const DevNum<T>& nm, int f, int F, int lane, T* Fm,
                                              T* sv, int stage_v, int* sr, int stage_r, T* v, T* scv)
{
    const int c0 = s.child_ptr[f], nch = s.child_ptr[f + 1] - c0;
    for (int k0 = 0; k0 < nch; k0 += 32) {
        int my_mc = 0, my_rel = 0;
        long long my_cb = 0;
        if (k0 + lane < nch) {
            const int ch = s.child_list[c0 + k0 + lane];
            my_mc = s.sn_front[ch] - (s.sn_first[ch + 1] - s.sn_first[ch]);
            my_cb = s.cb_off[ch];
            my_rel = s.rel_ptr[ch];
        }
        const int nb = min(32, nch - k0);
        // exclusive prefix sums over the lanes of mc^2 and mc
        int vx = my_mc * my_mc, rx = my_mc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int vu = __shfl_up_sync(kFull, vx, o), ru = __shfl_up_sync(kFull, rx, o);
            if (lane >= o) { vx += vu; rx += ru; }
        }
        vx -= my_mc * my_mc;
        rx -= my_mc;
        for (int k = 0; k < nb;) {
            const int vk = __shfl_sync(kFull, vx, k), rk = __shfl_sync(kFull, rx, k);
            // children k..k2-1 fit: prefix from k (sums grow with the lane)
            const bool fits = lane >= k && lane < nb && vx + my_mc * my_mc - vk <= stage_v &&
                              rx + my_mc - rk <= stage_r;
            const int k2 = k + __popc(__ballot_sync(kFull, fits));
            if (k2 == k) {                                            // too large: from global memory
                const int mc = __shfl_sync(kFull, my_mc, k);
                const T* cb = nm.cb + __shfl_sync(kFull, my_cb, k);
                const int relp = __shfl_sync(kFull, my_rel, k);
                const int rl = lane < mc ? s.rel[relp + lane] : 0;
                if (mc > 0) warp_add_child<T>(cb, mc, rl, F, lane, Fm);
                if (v && lane < mc) v[rl] += nm.cbv[relp + lane];      // forward step: the child's vector
                __syncwarp();
                ++k;
                continue;
            }
            for (int c = k; c < k2; ++c) {                            // every copy in flight together
                const int mc = __shfl_sync(kFull, my_mc, c);
                const T* cb = nm.cb + __shfl_sync(kFull, my_cb, c);
                const int relp = __shfl_sync(kFull, my_rel, c);
                const int vo = __shfl_sync(kFull, vx, c) - vk, ro = __shfl_sync(kFull, rx, c) - rk;
                for (int e = lane; e < mc * mc; e += 32) cp_async_word(sv + vo + e, cb + e, (int)sizeof(T));
                if (lane < mc) cp_async_word(sr + ro + lane, s.rel + relp + lane, 4);
                if (v && lane < mc) cp_async_word(scv + ro + lane, nm.cbv + relp + lane, (int)sizeof(T));
            }
            cp_async_wait_all();
            __syncwarp();
            for (int c = k; c < k2; ++c) {                            // in child order
                const int mc = __shfl_sync(kFull, my_mc, c);
                const int vo = __shfl_sync(kFull, vx, c) - vk, ro = __shfl_sync(kFull, rx, c) - rk;
                const int rl = lane < mc ? sr[ro + lane] : 0;
                if (mc > 0) warp_add_child<T>(sv + vo, mc, rl, F, lane, Fm);
                if (v && lane < mc) v[rl] += scv[ro + lane];
                __syncwarp();
            }
            k = k2;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(128, 8) front_warp_kernel(DevSched s, DevNum<T> nm0, const int* __restrict__ fronts,
                                                            int count, int maxF, int stage_v, int stage_r, int fused)
{
    // shared memory sized by the launch's largest front (maxF <= 32) and the
    // children's staging (per warp: stage_v values, stage_r relative
    // indices): the small leaf fronts of the widest levels keep many more
    // warps resident
    extern __shared__ __align__(16) unsigned char smraw[];
    const DevNum<T> nm = nm0.at(blockIdx.y);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int fi = blockIdx.x * 4 + wid;
    if (fi >= count) return;
    const int li = lane & 7, lj = lane >> 3;
    const int f = fronts[fi];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    // per warp: front (maxF^2), staged child blocks (stage_v), forward-step
    // vector (32) and staged child vectors (stage_r); then the indices
    T* Fm = reinterpret_cast<T*>(smraw) + (int64_t)wid * maxF * maxF;
    T* sv_base = reinterpret_cast<T*>(smraw) + (int64_t)4 * maxF * maxF;
    T* v = sv_base + (int64_t)4 * stage_v + wid * 32;
    T* scv = sv_base + (int64_t)4 * stage_v + 4 * 32 + (int64_t)wid * stage_r;
    int* sr_base = reinterpret_cast<int*>(sv_base + (int64_t)4 * (stage_v + 32 + stage_r));
    for (int t = lane; t < F * F; t += 32) Fm[t] = T(0);
    if (fused) v[lane] = lane < w ? nm.vec[first + lane] : T(0);  // F <= 32
    __syncwarp();
    assemble_original<T, 32>(s, nm, f, lane, Fm);
    __syncwarp();
    warp_children<T>(s, nm, f, F, lane, Fm, stage_v ? sv_base + (int64_t)wid * stage_v : nullptr, stage_v,
                     sr_base + wid * stage_r, stage_r, fused ? v : nullptr, scv);
    const T floorT = (T)(nm.pivot_eps * __longlong_as_double((long long)nm.stat->amax_bits));
    bool n_bad = false;
    int n_pert = 0;
    __shared__ T srinv[4];
    for (int p = 0; p < w; ++p) {                                 // one reciprocal per pivot
        if constexpr (sizeof(T) == 4) {
            T r;
            const T pv = uniform_pivot(Fm[p + p * F], floorT, r, n_bad, n_pert);
            __syncwarp();
            if (lane == 0) Fm[p + p * F] = pv;
            if (lane > p && lane < F) Fm[lane + p * F] *= r;
        } else {
            if (lane == 0) {
                const T pv = static_pivot(Fm[p + p * F], floorT, nm.stat, true);
                Fm[p + p * F] = pv;
                srinv[wid] = pivot_rcp(pv);
            }
            __syncwarp();
            if (lane > p && lane < F) Fm[lane + p * F] *= srinv[wid];
        }
        __syncwarp();
        for (int j = p + 1 + lj; j < F; j += 4) {
            const T u = Fm[p + j * F];
            for (int i = p + 1 + li; i < F; i += 8) Fm[i + j * F] -= Fm[i + p * F] * u;
        }
        __syncwarp();
    }
    if (lane == 0) count_pivot_events(nm.stat, n_bad, n_pert);
    if (fused) front_forward<T>(s, nm, f, first, w, F, Fm, v, lane, 32, kFull);
    T* pan = nm.panel + s.panel_off[f];
    const int m = F - w;
    for (int t = lane; t < F * w; t += 32) pan[t] = Fm[t];
    T* U12 = pan + F * w;                                          // column-major (ld = w)
    for (int b = lj; b < m; b += 4)
        for (int a = li; a < w; a += 8) U12[a + b * w] = Fm[a + (w + b) * F];
    T* cbo = nm.cb + s.cb_off[f];
    for (int b = lj; b < m; b += 4)
        for (int a = li; a < m; a += 8) cbo[a + b * m] = Fm[(w + a) + (w + b) * F];
}

// Childless fronts with F <= G (G = 8 or 16): G lanes per front, 32 / G
// fronts per warp, so the widest leaf level (tens of thousands of fronts of
// a handful of rows) needs a quarter or half of the warps, each going once
// through the same chain of dependent loads. Lanes of a group form 8 rows x
// G / 8 column groups; the arithmetic on every entry is that of
// front_warp_kernel (original entries, then one reciprocal and the rank-1
// updates per pivot, in pivot order); fused: the forward step of the
// right-hand side follows (childless: v starts as the pivot rows).
template <typename T, int G>
__global__ void __launch_bounds__(128) front_leaf_kernel(DevSched s, DevNum<T> nm0, const int* __restrict__ fronts,
                                                         int count, int fused)
{
    constexpr int NG = 32 / G, LJ = G / 8;
    __shared__ T Fall[4 * NG * G * G];
    __shared__ T Vall[4 * NG * G];                                 // fused: forward-step vectors
    __shared__ T srinv[4 * NG];                                    // double precision: the group's reciprocal
    const DevNum<T> nm = nm0.at(blockIdx.y);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gi = lane / G, gl = lane % G, slot = wid * NG + gi;
    const unsigned gmask = (unsigned)(((1ull << G) - 1ull) << (gi * G));
    const int fi = (blockIdx.x * 4 + wid) * NG + gi;
    if (fi >= count) return;                                       // the whole group
    const int li = gl & 7, lj = gl >> 3;
    const int f = fronts[fi];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    T* Fm = Fall + slot * G * G;                                   // leading dimension F <= G
    T* v = Vall + slot * G;
    for (int t = gl; t < F * F; t += G) Fm[t] = T(0);
    if (fused && gl < F) v[gl] = gl < w ? nm.vec[first + gl] : T(0);
    __syncwarp(gmask);
    assemble_original<T, G>(s, nm, f, gl, Fm);
    __syncwarp(gmask);
    const T floorT = (T)(nm.pivot_eps * __longlong_as_double((long long)nm.stat->amax_bits));
    bool n_bad = false;
    int n_pert = 0;
    for (int p = 0; p < w; ++p) {                                  // one reciprocal per pivot
        if constexpr (sizeof(T) == 4) {
            T r;
            const T pv = uniform_pivot(Fm[p + p * F], floorT, r, n_bad, n_pert);
            __syncwarp(gmask);
            if (gl == 0) Fm[p + p * F] = pv;
            if (gl > p && gl < F) Fm[gl + p * F] *= r;
        } else {
            if (gl == 0) {
                const T pv = static_pivot(Fm[p + p * F], floorT, nm.stat, true);
                Fm[p + p * F] = pv;
                srinv[slot] = pivot_rcp(pv);
            }
            __syncwarp(gmask);
            if (gl > p && gl < F) Fm[gl + p * F] *= srinv[slot];
        }
        __syncwarp(gmask);
        for (int j = p + 1 + lj; j < F; j += LJ) {
            const T u = Fm[p + j * F];
            for (int i = p + 1 + li; i < F; i += 8) Fm[i + j * F] -= Fm[i + p * F] * u;
        }
        __syncwarp(gmask);
    }
    if (gl == 0) count_pivot_events(nm.stat, n_bad, n_pert);
    if (fused) front_forward<T>(s, nm, f, first, w, F, Fm, v, gl, G, gmask);
    T* pan = nm.panel + s.panel_off[f];
    const int m = F - w;
    for (int t = gl; t < F * w; t += G) pan[t] = Fm[t];
    T* U12 = pan + F * w;                                          // column-major (ld = w)
    for (int b = lj; b < m; b += LJ)
        for (int a = li; a < w; a += 8) U12[a + b * w] = Fm[a + (w + b) * F];
    T* cbo = nm.cb + s.cb_off[f];
    for (int b = lj; b < m; b += LJ)
        for (int a = li; a < m; a += 8) cbo[a + b * m] = Fm[(w + a) + (w + b) * F];
}

// Fronts with F > 32 and a small contribution block: one CTA (8 warps) per
// front, the whole front in shared memory, right-looking rank-1 updates.
// Threads form a 32 x 8 grid: lane -> row, warp -> column.
template <typename T>
__global__ void __launch_bounds__(256) front_cta_kernel(DevSched s, DevNum<T> nm0, const int* __restrict__ fronts,
                                                        int count, int max_front)
{
    const DevNum<T> nm = nm0.at(blockIdx.y);
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Fm = reinterpret_cast<T*>(smraw);
    int* rls = reinterpret_cast<int*>(Fm + (int64_t)max_front * max_front);   // staged relative indices
    const int tid = threadIdx.x, nt = blockDim.x;
    const int tx = tid & 31, ty = tid >> 5;
    const int f = fronts[blockIdx.x];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    for (int t = tid; t < F * F; t += nt) Fm[t] = T(0);
    __syncthreads();
    assemble_original<T, 256>(s, nm, f, tid, Fm);
    __syncthreads();
    for (int c = s.child_ptr[f]; c < s.child_ptr[f + 1]; ++c) {
        const int ch = s.child_list[c];
        const int mc = s.sn_front[ch] - (s.sn_first[ch + 1] - s.sn_first[ch]);
        const T* cb = nm.cb + s.cb_off[ch];
        const int* rl = s.rel + s.rel_ptr[ch];
        for (int t = tid; t < mc; t += nt) rls[t] = rl[t];
        __syncthreads();
        for (int b = ty; b < mc; b += 8) {
            const int rb = rls[b] * F;
            for (int a = tx; a < mc; a += 32) Fm[rls[a] + rb] += cb[a + (int64_t)b * mc];
        }
        __syncthreads();
    }
    const T floorT = (T)(nm.pivot_eps * __longlong_as_double((long long)nm.stat->amax_bits));
    // single precision: every thread computes the pivot from the same entry
    // and the diagonal is written after the scaling barrier (nothing reads it
    // again in the loop); double precision: thread 0 computes it
    bool n_bad = false;
    int n_pert = 0;
    __shared__ T srinv;
    for (int p = 0; p < w; ++p) {                                 // one reciprocal per pivot
        if constexpr (sizeof(T) == 4) {
            T rinv;
            const T pv = uniform_pivot(Fm[p + p * F], floorT, rinv, n_bad, n_pert);
            for (int i = p + 1 + tid; i < F; i += nt) Fm[i + p * F] *= rinv;
            __syncthreads();
            if (tid == 0) Fm[p + p * F] = pv;
        } else {
            if (tid == 0) {
                const T pv = static_pivot(Fm[p + p * F], floorT, nm.stat, true);
                Fm[p + p * F] = pv;
                srinv = pivot_rcp(pv);
            }
            __syncthreads();
            const T rinv = srinv;
            for (int i = p + 1 + tid; i < F; i += nt) Fm[i + p * F] *= rinv;
            __syncthreads();
        }
        for (int j = p + 1 + ty; j < F; j += 8) {
            const T u = Fm[p + j * F];
            for (int i = p + 1 + tx; i < F; i += 32) Fm[i + j * F] -= Fm[i + p * F] * u;
        }
        __syncthreads();
    }
    if (tid == 0) count_pivot_events(nm.stat, n_bad, n_pert);
    T* pan = nm.panel + s.panel_off[f];
    const int m = F - w;
    for (int t = tid; t < F * w; t += nt) pan[t] = Fm[t];
    T* U12 = pan + F * w;                                          // column-major (ld = w)
    for (int b = ty; b < m; b += 8)
        for (int a = tx; a < w; a += 32) U12[a + b * w] = Fm[a + (w + b) * F];
    T* cbo = nm.cb + s.cb_off[f];
    for (int b = ty; b < m; b += 8)
        for (int a = tx; a < m; a += 32) cbo[a + b * m] = Fm[(w + a) + (w + b) * F];
}

// Fronts with a large contribution block. One CTA assembles the pivot panel
// (pivot columns F x w and pivot rows w x (F-w), in shared memory) -- all
// original entries fall there, and of each child's contribution block only
// the rows and columns that land on this front's pivots (a prefix, since
// relative indices increase) -- and factors the pivot columns (L11\U11, L21).
// The assembled pivot rows F12 go to scratch: schur_tile_kernel turns them into
// U12 = L11^{-1} F12 and updates the (2,2) block, spread over many CTAs.
template <typename T>
__global__ void __launch_bounds__(256) front_panel_kernel(DevSched s, DevNum<T> nm0, const int* __restrict__ fronts,
                                                          int count, T* gscratch, int64_t sstride)
{
    const DevNum<T> nm = nm0.at(blockIdx.y);
    extern __shared__ __align__(16) unsigned char smraw[];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int tx = tid & 31, ty = tid >> 5;
    const int f = fronts[blockIdx.x];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    const int m = F - w;
    T* col = gscratch ? gscratch + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * sstride
                      : reinterpret_cast<T*>(smraw);
    T* row = col + (int64_t)F * w;                                   // w x m, column-major (ld = w)
    for (int64_t t = tid; t < (int64_t)F * w + (int64_t)w * m; t += nt) col[t] = T(0);
    __syncthreads();
    {
        // original entries: position a + b*F of the full front; b < w -> pivot columns,
        // else a < w (entry (r, c) sits in the front of min(r, c)) -> pivot rows
        const int64_t e0 = s.asm_ptr[f], e1 = s.asm_ptr[f + 1];
        for (int64_t e = e0 + tid; e < e1; e += nt * 4) {
            int pos[4];
            T val[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t ee = e + nt * u;
                pos[u] = ee < e1 ? s.asm_pos[ee] : -1;
                val[u] = ee < e1 ? nm.sv[s.asm_src[ee]] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (pos[u] < 0) continue;
                if (pos[u] < F * w) col[pos[u]] = val[u];
                else {
                    const int rel = pos[u] - F * w;                 // a + (b - w) * F with a < w
                    const int bw = rel / F;                          // one division per original entry
                    row[(rel - bw * F) + (int64_t)bw * w] = val[u];
                }
            }
        }
    }
    __syncthreads();
    int* rls = gscratch ? nullptr : reinterpret_cast<int*>(row + (int64_t)w * m);
    for (int c = s.child_ptr[f]; c < s.child_ptr[f + 1]; ++c) {
        const int ch = s.child_list[c];
        const int mc = s.sn_front[ch] - (s.sn_first[ch + 1] - s.sn_first[ch]);
        const int k = s.cb_split[ch];
        if (k == 0) continue;
        const T* cb = nm.cb + s.cb_off[ch];
        const int* rl = s.rel + s.rel_ptr[ch];
        if (rls) {
            for (int t = tid; t < mc; t += nt) rls[t] = rl[t];
            __syncthreads();
            rl = rls;
        }
        // child columns j < k land on pivot columns: every row i
        for (int j = ty; j < k; j += 8) {
            const int64_t rj = (int64_t)rl[j] * F;
            for (int i = tx; i < mc; i += 32) col[rl[i] + rj] += cb[i + (int64_t)j * mc];
        }
        // child rows i < k, columns j >= k land on pivot rows, non-pivot columns
        for (int j = k + ty; j < mc; j += 8) {
            const int64_t rj = (int64_t)(rl[j] - w) * w;
            for (int i = tx; i < k; i += 32) row[rl[i] + rj] += cb[i + (int64_t)j * mc];
        }
        __syncthreads();
    }
    const T floorT = (T)(nm.pivot_eps * __longlong_as_double((long long)nm.stat->amax_bits));
    // single precision: every thread computes the pivot from the same entry
    // and the diagonal is written after the scaling barrier (nothing reads it
    // again in the loop); double precision: thread 0 computes it
    bool n_bad = false;
    int n_pert = 0;
    __shared__ T srinv;
    for (int p = 0; p < w; ++p) {                                 // one reciprocal per pivot
        if constexpr (sizeof(T) == 4) {
            T rinv;
            const T pv = uniform_pivot(col[p + (int64_t)p * F], floorT, rinv, n_bad, n_pert);
            for (int i = p + 1 + tid; i < F; i += nt) col[i + (int64_t)p * F] *= rinv;
            __syncthreads();
            if (tid == 0) col[p + (int64_t)p * F] = pv;
        } else {
            if (tid == 0) {
                const T pv = static_pivot(col[p + (int64_t)p * F], floorT, nm.stat, true);
                col[p + (int64_t)p * F] = pv;
                srinv = pivot_rcp(pv);
            }
            __syncthreads();
            const T rinv = srinv;
            for (int i = p + 1 + tid; i < F; i += nt) col[i + (int64_t)p * F] *= rinv;
            __syncthreads();
        }
        for (int j = p + 1 + ty; j < w; j += 8) {
            const T u = col[p + (int64_t)j * F];
            for (int i = p + 1 + tx; i < F; i += 32) col[i + (int64_t)j * F] -= col[i + (int64_t)p * F] * u;
        }
        __syncthreads();
    }
    if (tid == 0) count_pivot_events(nm.stat, n_bad, n_pert);
    T* pan = nm.panel + s.panel_off[f];
    for (int64_t t = tid; t < (int64_t)F * w; t += nt) pan[t] = col[t];
    T* f12 = nm.f12 + s.f12_off[f];
    for (int64_t t = tid; t < (int64_t)w * m; t += nt) f12[t] = row[t];
}

// One kTile x kTile tile (ti, tj) of a panel-class front's contribution block
// (kTile = 16: small tiles spread a narrow level over many SMs; one output
// per thread): solve L11 U = F12 for the tile's kTile columns of U12 (tiles
// of the first tile row store them), gather the children's contributions (in
// child order, through the gather maps), then C -= L21 U12 with the terms
// applied in pivot order, one fused multiply-add each, as the single-CTA
// kernels do.
template <typename T>
__global__ void __launch_bounds__(256) schur_tile_kernel(DevSched s, DevNum<T> nm0, const FrontTile* __restrict__ tiles,
                                                         int count)
{
    const DevNum<T> nm = nm0.at(blockIdx.y);
    static_assert(kTile * kTile == 256, "one output per thread");
    constexpr int KB = 64;
    constexpr int UL = kTile + 1;                                  // padded row length of the U12 tile
    __shared__ T Ls[KB][kTile + 1];
    __shared__ int gi[kTile], gj[kTile];
    extern __shared__ __align__(16) unsigned char smraw[];
    const FrontTile tl = tiles[blockIdx.x];
    const int f = tl.front;
    const int w = s.sn_first[f + 1] - s.sn_first[f];
    const int F = s.sn_front[f];
    const int m = F - w;
    const int i0 = tl.ti * kTile, j0 = tl.tj * kTile;
    const int tid = threadIdx.x;
    const int tx = tid & (kTile - 1), ty = tid / kTile;           // output (i0 + tx, j0 + ty)
    T* L11 = reinterpret_cast<T*>(smraw);                          // w x w, column-major
    T* Ut = L11 + w * w;                                           // w x kTile, row a at Ut[a * UL]
    T* pan = nm.panel + s.panel_off[f];
    const T* L21 = pan + w;                                        // row r, col p at L21[r + p*F]
    const T* F12 = nm.f12 + s.f12_off[f];                          // w x m, column-major
    for (int c = ty; c < w; c += 256 / kTile)
        for (int a = tx; a < w; a += kTile) L11[a + c * w] = pan[a + (int64_t)c * F];
    for (int c = ty; c < kTile; c += 256 / kTile)
        for (int a = tx; a < w; a += kTile) Ut[a * UL + c] = j0 + c < m ? F12[a + (int64_t)(j0 + c) * w] : T(0);
    __syncthreads();
    for (int p = 0; p + 1 < w; ++p) {                              // forward substitution, unit L11
        for (int a = p + 1 + ty; a < w; a += 256 / kTile) Ut[a * UL + tx] -= L11[a + p * w] * Ut[p * UL + tx];
        __syncthreads();
    }
    if (tl.ti == 0) {
        T* U12 = pan + (int64_t)F * w;                             // row p, col c at U12[p + c*w]
        for (int c = ty; c < kTile; c += 256 / kTile)
            for (int a = tx; a < w; a += kTile)
                if (j0 + c < m) U12[a + (int64_t)(j0 + c) * w] = Ut[a * UL + c];
    }
    T* C = nm.cb + s.cb_off[f];
    const int i = i0 + tx, j = j0 + ty;
    T acc = T(0);
    const int* inv = s.inv + s.inv_off[f];
    for (int c = s.child_ptr[f]; c < s.child_ptr[f + 1]; ++c, inv += m) {
        const int ch = s.child_list[c];
        const int mc = s.sn_front[ch] - (s.sn_first[ch + 1] - s.sn_first[ch]);
        const T* cb = nm.cb + s.cb_off[ch];
        __syncthreads();
        if (tid < kTile) gi[tid] = i0 + tid < m ? inv[i0 + tid] : -1;
        else if (tid < 2 * kTile) gj[tid - kTile] = j0 + tid - kTile < m ? inv[j0 + tid - kTile] : -1;
        __syncthreads();
        const int a = gi[tx], b = gj[ty];
        if (a >= 0 && b >= 0) acc += cb[a + (int64_t)b * mc];
    }
    for (int p0 = 0; p0 < w; p0 += KB) {
        const int kb = min(KB, w - p0);
        __syncthreads();
        for (int c = ty; c < kb; c += 256 / kTile)
            Ls[c][tx] = i0 + tx < m ? L21[(i0 + tx) + (int64_t)(p0 + c) * F] : T(0);
        __syncthreads();
        for (int c = 0; c < kb; ++c) acc -= Ls[c][tx] * Ut[(p0 + c) * UL + ty];
    }
    if (i < m && j < m) C[i + (int64_t)j * m] = acc;
}

// ------------------------------------------------------------ solve kernels

template <typename T>
__global__ void solve_pre_kernel(int n, const int* __restrict__ perm, DevNum<T> nm0, const double* __restrict__ b)
{
    const DevNum<T> nm = nm0.at(blockIdx.y);
    const double* __restrict__ d = nm.d;
    T* __restrict__ vec = nm.vec;
    b += (int64_t)blockIdx.y * n;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        int o = perm[k];
        vec[k] = (T)(d[o] * b[o]);
    }
}

template <typename T>
__global__ void solve_post_kernel(int n, const int* __restrict__ perm, DevNum<T> nm0, double* __restrict__ x)
{
    const DevNum<T> nm = nm0.at(blockIdx.y);
    const double* __restrict__ d = nm.d;
    const T* __restrict__ vec = nm.vec;
    x += (int64_t)blockIdx.y * n;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        int o = perm[k];
        x[o] = d[o] * (double)vec[k];
    }
}

// Back substitution with the upper pivot block U (column-major, leading
// dimension w <= G, in shared memory) by a group of G lanes (gmask, lane gl
// of the group holding v_gl in a register, the pivot entry broadcast by a
// shuffle); the operations and their order are those of the shared-memory
// loop x_p = v_p * (1 / u_pp), v_a -= u_ap x_p (the bits are the same). FP64
// costs pipe time per active lane, so the reciprocals are formed by all lanes
// at once before the dependent chain, and on the chain each step is one
// lane's multiply and the FMAs of the lanes above the pivot (instead of a
// reciprocal and a multiply on every lane per step: 0.184 -> 0.165 ms of
// solve_bwd_kernel per 70k FP64 solve). A register version of the forward
// block was slower on the wide levels (more instructions per front) and is
// not used there.
template <typename T, int G>
__device__ __forceinline__ void group_pivot_upper(T* v, const T* U, int w, unsigned gmask, int gl)
{
    T x = gl < w ? v[gl] : T(0);
    const T r = gl < w ? pivot_rcp(U[gl + gl * w]) : T(0);
    T ua[G];
#pragma unroll
    for (int p = 0; p < G; ++p) ua[p] = (p < w && gl < w) ? U[gl + p * w] : T(0);
#pragma unroll
    for (int p = G - 1; p >= 0; --p) {
        if (p >= w) continue;
        if (gl == p) x *= r;                                       // x_p = v_p * (1 / u_pp)
        const T xp = __shfl_sync(gmask, x, p, G);
        if (gl < p) x -= ua[p] * xp;
    }
    if (gl < w) v[gl] = x;
    __syncwarp(gmask);
}

// Forward substitution y = L^{-1} c, multifrontally: one warp per front
// gathers its pivot entries and its children's contribution vectors, solves
// with its unit lower pivot block (staged in shared memory), then updates its
// other rows with L21 (lane per row, coalesced column reads) and leaves them as
// its own contribution vector.
template <typename T>
__global__ void __launch_bounds__(128) solve_fwd_kernel(DevSched s, DevNum<T> nm0, const int* __restrict__ fronts,
                                                        int count, int max_front, int max_w)
{
    const DevNum<T> nm = nm0.at(blockIdx.y);
    extern __shared__ __align__(16) unsigned char smraw[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int fi = blockIdx.x * 4 + wid;
    if (fi >= count) return;
    T* v = reinterpret_cast<T*>(smraw) + (int64_t)wid * (max_front + max_w * max_w);
    T* Ls = v + max_front;
    const int f = fronts[fi];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    const T* pan = nm.panel + s.panel_off[f];
    for (int a = lane; a < F; a += 32) v[a] = a < w ? nm.vec[first + a] : T(0);
    for (int c = lane >> 3; c < w; c += 4)
        for (int a = lane & 7; a < w; a += 8) Ls[a + c * w] = pan[a + (int64_t)c * F];
    __syncwarp();
    for (int c = s.child_ptr[f]; c < s.child_ptr[f + 1]; ++c) {
        const int ch = s.child_list[c];
        const int mc = s.sn_front[ch] - (s.sn_first[ch + 1] - s.sn_first[ch]);
        const T* cv = nm.cbv + s.rel_ptr[ch];
        const int* rl = s.rel + s.rel_ptr[ch];
        for (int t = lane; t < mc; t += 32) v[rl[t]] += cv[t];
        __syncwarp();
    }
    for (int p = 0; p < w; ++p) {
        const T xp = v[p];
        for (int i = p + 1 + lane; i < w; i += 32) v[i] -= Ls[i + p * w] * xp;
        __syncwarp();
    }
    for (int i = w + lane; i < F; i += 32) {
        T acc = v[i];
        for (int p = 0; p < w; ++p) acc -= pan[i + (int64_t)p * F] * v[p];
        v[i] = acc;
    }
    __syncwarp();
    for (int a = lane; a < w; a += 32) nm.vec[first + a] = v[a];
    T* cv = nm.cbv + s.rel_ptr[f];
    for (int t = lane; t < F - w; t += 32) cv[t] = v[w + t];
}

// Back substitution x = U^{-1} y, top-down: one warp per front gathers the
// already known solution entries of its other rows, subtracts U12 x (lane per
// pivot row, coalesced reads of the column-major U12), and back-substitutes
// with its upper pivot block staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(128) solve_bwd_kernel(DevSched s, DevNum<T> nm0, const int* __restrict__ fronts,
                                                        int count, int max_front, int max_w)
{
    const DevNum<T> nm = nm0.at(blockIdx.y);
    extern __shared__ __align__(16) unsigned char smraw[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int fi = blockIdx.x * 4 + wid;
    if (fi >= count) return;
    T* v = reinterpret_cast<T*>(smraw) + (int64_t)wid * (max_front + max_w * max_w);
    T* Us = v + max_front;
    const int f = fronts[fi];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    const int m = F - w;
    const int* R = s.rows + s.rows_ptr[f];
    const T* pan = nm.panel + s.panel_off[f];
    const T* U12 = pan + (int64_t)F * w;
    for (int t = lane; t < m; t += 32) v[w + t] = nm.vec[R[w + t]];
    for (int c = lane >> 3; c < w; c += 4)
        for (int a = lane & 7; a < w; a += 8) Us[a + c * w] = pan[a + (int64_t)c * F];
    __syncwarp();
    // y_a - sum_t U12[a, t] x_t in sequence (m < 32 <= kSeqSum here: the order every backward kernel uses)
    for (int a = lane; a < w; a += 32) {
        T acc = nm.vec[first + a];
        for (int t = 0; t < m; ++t) acc -= U12[a + (int64_t)t * w] * v[w + t];
        v[a] = acc;
    }
    __syncwarp();
    if (w <= 32)
        group_pivot_upper<T, 32>(v, Us, w, 0xffffffffu, lane);
    else
        for (int p = w - 1; p >= 0; --p) {
            const T xp = v[p] * pivot_rcp(Us[p + p * w]);    // x_p = v_p * (1 / u_pp), as every backward kernel
            __syncwarp();
            if (lane == 0) v[p] = xp;
            for (int a = lane; a < p; a += 32) v[a] -= Us[a + p * w] * xp;
            __syncwarp();
        }
    for (int a = lane; a < w; a += 32) nm.vec[first + a] = v[a];
}

// Back substitution of childless fronts with F <= G (G = 8 or 16): G lanes per
// front, 32 / G fronts per warp (the widest leaf level), the operations of
// solve_bwd_kernel in its order.
template <typename T, int G>
__global__ void __launch_bounds__(128) solve_bwd_leaf_kernel(DevSched s, DevNum<T> nm0, const int* __restrict__ fronts,
                                                             int count)
{
    constexpr int NG = 32 / G;
    __shared__ T Vall[4 * NG * G];
    __shared__ T Uall[4 * NG * G * G];
    const DevNum<T> nm = nm0.at(blockIdx.y);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gi = lane / G, gl = lane % G, slot = wid * NG + gi;
    const unsigned gmask = (unsigned)(((1ull << G) - 1ull) << (gi * G));
    const int fi = (blockIdx.x * 4 + wid) * NG + gi;
    if (fi >= count) return;                                       // the whole group
    T* v = Vall + slot * G;
    T* Us = Uall + slot * G * G;
    const int f = fronts[fi];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    const int m = F - w;
    const int* R = s.rows + s.rows_ptr[f];
    const T* pan = nm.panel + s.panel_off[f];
    const T* U12 = pan + (int64_t)F * w;
    for (int t = gl; t < m; t += G) v[w + t] = nm.vec[R[w + t]];
    for (int e = gl; e < w * w; e += G) {
        const int c = e / w, a = e - c * w;
        Us[a + c * w] = pan[a + (int64_t)c * F];
    }
    __syncwarp(gmask);
    for (int a = gl; a < w; a += G) {
        T acc = nm.vec[first + a];
        for (int t = 0; t < m; ++t) acc -= U12[a + (int64_t)t * w] * v[w + t];
        v[a] = acc;
    }
    __syncwarp(gmask);
    group_pivot_upper<T, G>(v, Us, w, gmask, gl);                  // w <= F <= G
    for (int a = gl; a < w; a += G) nm.vec[first + a] = v[a];
}

// The same two substitutions for larger fronts, one CTA (128 threads) per
// front: one warp does the sequential pivot block, all threads the L21 / U12
// products.
template <typename T>
__global__ void __launch_bounds__(128) solve_fwd_cta_kernel(DevSched s, DevNum<T> nm0, const int* __restrict__ fronts,
                                                            int count, int max_front, int max_w)
{
    const DevNum<T> nm = nm0.at(blockIdx.y);
    extern __shared__ __align__(16) unsigned char smraw[];
    const int tid = threadIdx.x, lane = tid & 31;
    T* v = reinterpret_cast<T*>(smraw);
    T* Ls = v + max_front;
    const int f = fronts[blockIdx.x];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    const T* pan = nm.panel + s.panel_off[f];
    for (int a = tid; a < F; a += 128) v[a] = a < w ? nm.vec[first + a] : T(0);
    for (int c = tid >> 5; c < w; c += 4)
        for (int a = lane; a < w; a += 32) Ls[a + c * w] = pan[a + (int64_t)c * F];
    __syncthreads();
    for (int c = s.child_ptr[f]; c < s.child_ptr[f + 1]; ++c) {
        const int ch = s.child_list[c];
        const int mc = s.sn_front[ch] - (s.sn_first[ch + 1] - s.sn_first[ch]);
        const T* cv = nm.cbv + s.rel_ptr[ch];
        const int* rl = s.rel + s.rel_ptr[ch];
        for (int t = tid; t < mc; t += 128) v[rl[t]] += cv[t];
        __syncthreads();
    }
    if (tid < 32) {
        for (int p = 0; p < w; ++p) {
            const T xp = v[p];
            for (int i = p + 1 + lane; i < w; i += 32) v[i] -= Ls[i + p * w] * xp;
            __syncwarp();
        }
    }
    __syncthreads();
    for (int i = w + tid; i < F; i += 128) {
        T acc = v[i];
        for (int p = 0; p < w; ++p) acc -= pan[i + (int64_t)p * F] * v[p];
        v[i] = acc;
    }
    __syncthreads();
    for (int a = tid; a < w; a += 128) nm.vec[first + a] = v[a];
    T* cv = nm.cbv + s.rel_ptr[f];
    for (int t = tid; t < F - w; t += 128) cv[t] = v[w + t];
}

template <typename T>
__global__ void __launch_bounds__(128) solve_bwd_cta_kernel(DevSched s, DevNum<T> nm0, const int* __restrict__ fronts,
                                                            int count, int max_front, int max_w)
{
    const DevNum<T> nm = nm0.at(blockIdx.y);
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ T red[128];
    const int tid = threadIdx.x, lane = tid & 31;
    T* v = reinterpret_cast<T*>(smraw);
    T* Us = v + max_front;
    const int f = fronts[blockIdx.x];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    const int m = F - w;
    const int* R = s.rows + s.rows_ptr[f];
    const T* pan = nm.panel + s.panel_off[f];
    const T* U12 = pan + (int64_t)F * w;
    for (int t = tid; t < m; t += 128) v[w + t] = nm.vec[R[w + t]];
    for (int c = tid >> 5; c < w; c += 4)
        for (int a = lane; a < w; a += 32) Us[a + c * w] = pan[a + (int64_t)c * F];
    __syncthreads();
    // y_a - sum_t U12[a, t] x_t: in sequence for m <= kSeqSum, else thread (a, g)
    // sums every G-th t and the row sums are added in g order (the order every
    // backward kernel uses)
    if (m <= kSeqSum) {
        for (int a = tid; a < w; a += 128) {
            T acc = nm.vec[first + a];
            for (int t = 0; t < m; ++t) acc -= U12[a + (int64_t)t * w] * v[w + t];
            v[a] = acc;
        }
    } else {
        const int G = 128 / w;
        T part = T(0);
        if (tid < G * w) {
            const int a = tid % w, g = tid / w;
            for (int t = g; t < m; t += G) part += U12[a + (int64_t)t * w] * v[w + t];
        }
        red[tid] = part;
        __syncthreads();
        for (int a = tid; a < w; a += 128) {
            T acc = T(0);
            for (int g = 0; g < G; ++g) acc += red[a + g * w];
            v[a] = nm.vec[first + a] - acc;
        }
    }
    __syncthreads();
    if (tid < 32) {
        if (w <= 32)
            group_pivot_upper<T, 32>(v, Us, w, 0xffffffffu, lane);
        else
            for (int p = w - 1; p >= 0; --p) {
                const T xp = v[p] * pivot_rcp(Us[p + p * w]);    // x_p = v_p * (1 / u_pp), as every backward kernel
                __syncwarp();
                if (lane == 0) v[p] = xp;
                for (int a = lane; a < p; a += 32) v[a] -= Us[a + p * w] * xp;
                __syncwarp();
            }
    }
    __syncthreads();
    for (int a = tid; a < w; a += 128) nm.vec[first + a] = v[a];
}

// ---------------------------------------------------------- FP64 vectors

// y = b - K x (b != nullptr) or y = K x on the sliced copy of K, a lane per
// row summing its entries in CSR order.
__global__ void __launch_bounds__(256) spmv_sell_kernel(DevSched s, const double* __restrict__ kv,
                                                        const double* __restrict__ x, const double* __restrict__ b,
                                                        double* __restrict__ y)
{
    const int lane = threadIdx.x & 31;
    const int slice = blockIdx.x * kSellWarps + (threadIdx.x >> 5);
    if (slice >= s.nslices) return;
    const int row = s.sell_row[slice * 32 + lane];
    const double acc = sell_row_dot(s, kv, x, s.sell_off[slice] + lane, s.sell_off[slice + 1]);
    if (row >= 0) y[row] = b ? b[row] - acc : acc;
}

constexpr int kRedBlocks = 304;   // 2 x 152 SMs

// partial dot products of nv vectors with w: part[blk * nv + k]
__global__ void multidot_part_kernel(int n, const double* __restrict__ V, int64_t ldv, int nv,
                                     const double* __restrict__ w, double* __restrict__ part)
{
    extern __shared__ double red[];     // nv * (blockDim/32)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < nv; ++k) {
        double s = 0.0;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
            s += V[i + (int64_t)k * ldv] * w[i];
        s = warp_sum(s);
        if (lane == 0) red[k * nw + wid] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < nw; ++q) s += red[k * nw + q];
        part[(int64_t)blockIdx.x * nv + k] = s;
    }
}

__global__ void multidot_final_kernel(int nblk, int nv, const double* __restrict__ part, double* __restrict__ out)
{
    const int k = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) s += part[(int64_t)b * nv + k];
    s = warp_sum(s);
    if (threadIdx.x == 0) out[k] = s;
}

__global__ void multiaxpy_kernel(int n, double* __restrict__ w, const double* __restrict__ V, int64_t ldv, int nv,
                                 const double* __restrict__ h)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = w[i];
        for (int k = 0; k < nv; ++k) acc -= V[i + (int64_t)k * ldv] * h[k];
        w[i] = acc;
    }
}

__global__ void update_kernel(int n, double* __restrict__ x, const double* __restrict__ Z, int64_t ldz, int nv,
                              const double* __restrict__ y)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = x[i];
        for (int k = 0; k < nv; ++k) acc += Z[i + (int64_t)k * ldz] * y[k];
        x[i] = acc;
    }
}

__global__ void scal_copy_kernel(int n, const double* __restrict__ x, double* __restrict__ y,
                                 const double* __restrict__ alpha, int invert)
{
    const double a = invert ? 1.0 / *alpha : *alpha;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = x[i] * a;
}

// FGMRES, step j of the Arnoldi process, on the device: column j of the
// Hessenberg matrix (h1 already stored in it, h2 added here), its subdiagonal
// entry h_{j+1,j} = ||w||_2, the earlier Givens rotations applied to the
// column, the new rotation that zeroes h_{j+1,j}, and the rotated right-hand
// side g. scale receives h_{j+1,j} (the next basis vector is w / scale);
// flag[j] = 1 once |g_{j+1}| <= target, on breakdown (h_{j+1,j} = 0) or on a
// non-finite value. One thread: the rotations are a chain of dependent steps.
__global__ void fgmres_givens_kernel(int j, int ldh, const double* __restrict__ h2, const double* __restrict__ nrm,
                                     double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                                     double* __restrict__ g, double* __restrict__ scale, double* __restrict__ flag,
                                     double target)
{
    if (threadIdx.x != 0) return;
    double* col = H + (int64_t)j * ldh;
    for (int i = 0; i <= j; ++i) col[i] += h2[i];
    const double hn = sqrt(nrm[1]);
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
    }
    const double a = col[j], b = col[j + 1];
    const double rho = sqrt(a * a + b * b);
    cs[j] = rho > 0.0 ? a / rho : 1.0;
    sn[j] = rho > 0.0 ? b / rho : 0.0;
    col[j] = rho;
    col[j + 1] = 0.0;
    const double gj = g[j];
    g[j + 1] = -sn[j] * gj;
    g[j] = cs[j] * gj;
    *scale = hn;
    flag[j] = (fabs(g[j + 1]) <= target || hn == 0.0 || !isfinite(g[j + 1])) ? 1.0 : 0.0;
}

// Start of an FGMRES cycle: g = (beta, 0, ..., 0), scale = beta.
__global__ void fgmres_start_kernel(int m, double beta, double* __restrict__ g, double* __restrict__ scale)
{
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = i == 0 ? beta : 0.0;
    if (threadIdx.x == 0) *scale = beta;
}

// y = R^-1 g over the first k rows and columns of the rotated Hessenberg
// matrix (upper triangular), by back substitution; one warp, each lane summing
// the products of every 32nd column.
__global__ void fgmres_lsq_kernel(int k, int ldh, const double* __restrict__ H, const double* __restrict__ g,
                                  double* y)
{
    const int lane = threadIdx.x & 31;
    for (int i = k - 1; i >= 0; --i) {
        double part = 0.0;
        for (int t = i + 1 + lane; t < k; t += 32) part += H[i + (int64_t)t * ldh] * y[t];
        part = warp_sum(part);
        if (lane == 0) y[i] = (g[i] - part) / H[i + (int64_t)i * ldh];
        __syncwarp();
    }
}

// ||a||_inf and ||a||_2^2. The maximum is taken on the bit patterns of |a_i|
// (the numeric order for non-negative doubles, with NaN above +Inf), so a NaN
// entry makes the norm NaN instead of being dropped.
__global__ void norms_part_kernel(int n, const double* __restrict__ a, double* __restrict__ part)
{
    __shared__ unsigned long long smax[32];
    __shared__ double ssum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long mx = 0ull;
    double sq = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = a[i];
        mx = umax64(mx, abs_bits(v));
        sq += v * v;
    }
    mx = warp_umax(mx);
    sq = warp_sum(sq);
    if (lane == 0) { smax[wid] = mx; ssum[wid] = sq; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long M = 0ull;
        double S = 0.0;
        for (int q = 0; q < nw; ++q) { M = umax64(M, smax[q]); S += ssum[q]; }
        part[2 * blockIdx.x] = __longlong_as_double((long long)M);
        part[2 * blockIdx.x + 1] = S;
    }
}

__global__ void norms_final_kernel(int nblk, const double* __restrict__ part, double* __restrict__ out)
{
    unsigned long long M = 0ull;
    double S = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) {
        M = umax64(M, (unsigned long long)__double_as_longlong(part[2 * b]));
        S += part[2 * b + 1];
    }
    M = warp_umax(M);
    S = warp_sum(S);
    if (threadIdx.x == 0) { out[0] = __longlong_as_double((long long)M); out[1] = S; }
}

}  // namespace

// ================================================================ launchers

static inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

cudaError_t launch_zero_stat(DevStat* stat, cudaStream_t st)
{
    return cudaMemsetAsync(stat, 0, sizeof(DevStat), st);
}

static inline int sell_blocks(const DevSched& s) { return cdiv(s.nslices, kSellWarps); }

cudaError_t launch_ruiz(const DevSched& s, const double* vals, int64_t bs_nnz, double* kcopy, unsigned short* keys,
                        int64_t bs_slot, double* d, double* dtmp, int iters, DevStat* stat, double** d_final,
                        int batch, cudaStream_t st)
{
    const dim3 grid(sell_blocks(s), batch);
    double* a = d;
    double* b = dtmp;
    if (iters == 0) {
        ruiz_sell_kernel<<<grid, 256, 0, st>>>(s, vals, bs_nnz, kcopy, keys, bs_slot, a, b, stat, 0, 1);
        *d_final = a;
        return cudaGetLastError();
    }
    for (int it = 0; it < iters; ++it) {
        ruiz_sell_kernel<<<grid, 256, 0, st>>>(s, vals, bs_nnz, kcopy, keys, bs_slot, a, b, stat, it, 0);
        double* t = a; a = b; b = t;
    }
    *d_final = a;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale(const DevSched& s, const DevNum<T>& nm, const double* d, int batch, cudaStream_t st)
{
    (void)d;
    scale_sell_kernel<T><<<dim3(sell_blocks(s), batch), 256, 0, st>>>(s, nm);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fronts_warp(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, int max_front,
                               int stage_v, int stage_r, int fused, int batch, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    if (max_front < 1 || max_front > kWarpFrontMax || stage_v < 0 || stage_r < 0) return cudaErrorInvalidValue;
    const size_t smem = 4 * ((size_t)(max_front * max_front + stage_v + 32 + stage_r) * sizeof(T) +
                             (size_t)stage_r * sizeof(int));
    front_warp_kernel<T><<<dim3(cdiv(count, 4), batch), 128, smem, st>>>(s, nm, fronts, count, max_front, stage_v,
                                                                         stage_r, fused);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fronts_leaf(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, int group,
                               int fused, int batch, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    if (group == 8)
        front_leaf_kernel<T, 8><<<dim3(cdiv(count, 16), batch), 128, 0, st>>>(s, nm, fronts, count, fused);
    else if (group == 16)
        front_leaf_kernel<T, 16><<<dim3(cdiv(count, 8), batch), 128, 0, st>>>(s, nm, fronts, count, fused);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_bwd_leaf(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, int group,
                                  int batch, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    if (group == 8)
        solve_bwd_leaf_kernel<T, 8><<<dim3(cdiv(count, 16), batch), 128, 0, st>>>(s, nm, fronts, count);
    else if (group == 16)
        solve_bwd_leaf_kernel<T, 16><<<dim3(cdiv(count, 8), batch), 128, 0, st>>>(s, nm, fronts, count);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fronts_cta(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, int max_front,
                              int batch, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    size_t smem = (size_t)max_front * max_front * sizeof(T) + (size_t)max_front * sizeof(int);
    front_cta_kernel<T><<<dim3(count, batch), 256, smem, st>>>(s, nm, fronts, count, max_front);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fronts_panel(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count,
                                size_t smem_bytes, T* gscratch, int64_t scratch_stride, int batch, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    front_panel_kernel<T><<<dim3(count, batch), 256, gscratch ? 0 : smem_bytes, st>>>(s, nm, fronts, count, gscratch,
                                                                                      scratch_stride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_schur_tiles(const DevSched& s, const DevNum<T>& nm, const FrontTile* tiles, int count,
                               int max_w, int batch, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = (size_t)(max_w * max_w + max_w * (kTile + 1)) * sizeof(T);
    schur_tile_kernel<T><<<dim3(count, batch), 256, smem, st>>>(s, nm, tiles, count);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_pre(const DevSched& s, const DevNum<T>& nm, const double* b, int batch, cudaStream_t st)
{
    solve_pre_kernel<T><<<dim3(cdiv(s.n, 256), batch), 256, 0, st>>>(s.n, s.perm, nm, b);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_post(const DevSched& s, const DevNum<T>& nm, double* x, int batch, cudaStream_t st)
{
    solve_post_kernel<T><<<dim3(cdiv(s.n, 256), batch), 256, 0, st>>>(s.n, s.perm, nm, x);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_fwd(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, int max_front,
                             int max_w, int batch, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = 4 * (size_t)(max_front + max_w * max_w) * sizeof(T);
    solve_fwd_kernel<T><<<dim3(cdiv(count, 4), batch), 128, smem, st>>>(s, nm, fronts, count, max_front, max_w);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_bwd(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, int max_front,
                             int max_w, int batch, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = 4 * (size_t)(max_front + max_w * max_w) * sizeof(T);
    solve_bwd_kernel<T><<<dim3(cdiv(count, 4), batch), 128, smem, st>>>(s, nm, fronts, count, max_front, max_w);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_fwd_cta(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, int max_front,
                                 int max_w, int batch, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = (size_t)(max_front + max_w * max_w) * sizeof(T);
    solve_fwd_cta_kernel<T><<<dim3(count, batch), 128, smem, st>>>(s, nm, fronts, count, max_front, max_w);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_bwd_cta(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, int max_front,
                                 int max_w, int batch, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = (size_t)(max_front + max_w * max_w) * sizeof(T);
    solve_bwd_cta_kernel<T><<<dim3(count, batch), 128, smem, st>>>(s, nm, fronts, count, max_front, max_w);
    return cudaGetLastError();
}

cudaError_t launch_spmv_resid(const DevSched& s, const double* kv, const double* x, const double* b, double* r,
                              cudaStream_t st)
{
    spmv_sell_kernel<<<sell_blocks(s), 256, 0, st>>>(s, kv, x, b, r);
    return cudaGetLastError();
}

cudaError_t launch_spmv(const DevSched& s, const double* kv, const double* x, double* y, cudaStream_t st)
{
    spmv_sell_kernel<<<sell_blocks(s), 256, 0, st>>>(s, kv, x, nullptr, y);
    return cudaGetLastError();
}

// The partial sums need a scratch area: it lives right after `out` in a
// buffer the caller sized with multidot_scratch_doubles().
cudaError_t launch_multidot(int n, const double* V, int64_t ldv, int nv, const double* w, double* out,
                            cudaStream_t st)
{
    double* part = out + 128;
    int blocks = kRedBlocks;
    multidot_part_kernel<<<blocks, 256, (size_t)nv * 8 * sizeof(double), st>>>(n, V, ldv, nv, w, part);
    multidot_final_kernel<<<nv, 32, 0, st>>>(blocks, nv, part, out);
    return cudaGetLastError();
}

cudaError_t launch_multiaxpy(int n, double* w, const double* V, int64_t ldv, int nv, const double* h,
                             cudaStream_t st)
{
    multiaxpy_kernel<<<kRedBlocks, 256, 0, st>>>(n, w, V, ldv, nv, h);
    return cudaGetLastError();
}

cudaError_t launch_scal_copy(int n, const double* x, double* y, const double* alpha, int invert, cudaStream_t st)
{
    scal_copy_kernel<<<kRedBlocks, 256, 0, st>>>(n, x, y, alpha, invert);
    return cudaGetLastError();
}

cudaError_t launch_update(int n, double* x, const double* Z, int64_t ldz, int nv, const double* y, cudaStream_t st)
{
    update_kernel<<<kRedBlocks, 256, 0, st>>>(n, x, Z, ldz, nv, y);
    return cudaGetLastError();
}

cudaError_t launch_fgmres_givens(int j, int ldh, const double* h2, const double* nrm, double* H, double* cs,
                                 double* sn, double* g, double* scale, double* flag, double target, cudaStream_t st)
{
    fgmres_givens_kernel<<<1, 32, 0, st>>>(j, ldh, h2, nrm, H, cs, sn, g, scale, flag, target);
    return cudaGetLastError();
}

cudaError_t launch_fgmres_start(int m, double beta, double* g, double* scale, cudaStream_t st)
{
    fgmres_start_kernel<<<1, 128, 0, st>>>(m, beta, g, scale);
    return cudaGetLastError();
}

cudaError_t launch_fgmres_lsq(int k, int ldh, const double* H, const double* g, double* y, cudaStream_t st)
{
    fgmres_lsq_kernel<<<1, 32, 0, st>>>(k, ldh, H, g, y);
    return cudaGetLastError();
}

cudaError_t launch_norms(int n, const double* a, double* out, cudaStream_t st)
{
    double* part = out + 2;
    norms_part_kernel<<<kRedBlocks, 256, 0, st>>>(n, a, part);
    norms_final_kernel<<<1, 32, 0, st>>>(kRedBlocks, part, out);
    return cudaGetLastError();
}

// Batched residual and backward error: grid (slice blocks, batch), a lane per
// row on the sliced copy of K. Maxima of non-negative doubles are taken on
// their bit patterns (integer pipes; NaN sorts above +Inf, so it reaches
// omega); ||K||_inf comes from the refactorization's statistics. Each block
// stores max |r|, |x|, |b| of its rows (as bits) in its slot of `part`;
// omega_final_batched reduces the slots.
__global__ void __launch_bounds__(256) resid_omega_part_kernel(DevSched s, const double* __restrict__ kv,
                                                               int64_t bs_slot, const double* __restrict__ x,
                                                               const double* __restrict__ b, double* __restrict__ r,
                                                               unsigned long long* __restrict__ part)
{
    __shared__ unsigned long long red[3][kSellWarps];
    const int inst = blockIdx.y;
    const int n = s.n;
    kv += (int64_t)inst * bs_slot;
    x += (int64_t)inst * n;
    b += (int64_t)inst * n;
    r += (int64_t)inst * n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int slice = blockIdx.x * kSellWarps + wid;
    unsigned long long mr = 0ull, mx = 0ull, mb = 0ull;
    if (slice < s.nslices) {
        const int row = s.sell_row[slice * 32 + lane];
        const double acc = sell_row_dot(s, kv, x, s.sell_off[slice] + lane, s.sell_off[slice + 1]);
        if (row >= 0) {
            const double ri = b[row] - acc;
            r[row] = ri;
            mr = abs_bits(ri);
            mx = abs_bits(x[row]);
            mb = abs_bits(b[row]);
        }
    }
    mr = warp_umax(mr); mx = warp_umax(mx); mb = warp_umax(mb);
    if (lane == 0) { red[0][wid] = mr; red[1][wid] = mx; red[2][wid] = mb; }
    __syncthreads();
    if (threadIdx.x < 3) {
        unsigned long long m = 0ull;
        for (int q = 0; q < kSellWarps; ++q) m = umax64(m, red[threadIdx.x][q]);
        part[((int64_t)inst * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = m;
    }
}

__global__ void __launch_bounds__(256) omega_final_batched_kernel(int nblk, const unsigned long long* __restrict__ part,
                                                                  const DevStat* __restrict__ stat,
                                                                  double* __restrict__ omega)
{
    __shared__ unsigned long long red[3][8];
    const int inst = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long* pp = part + (int64_t)inst * nblk * 4;
    unsigned long long mr = 0ull, mx = 0ull, mb = 0ull;
    for (int i = threadIdx.x; i < nblk; i += 256) {
        mr = umax64(mr, pp[4 * i + 0]);
        mx = umax64(mx, pp[4 * i + 1]);
        mb = umax64(mb, pp[4 * i + 2]);
    }
    mr = warp_umax(mr); mx = warp_umax(mx); mb = warp_umax(mb);
    if (lane == 0) { red[0][wid] = mr; red[1][wid] = mx; red[2][wid] = mb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < 8; ++q) {
            red[0][0] = umax64(red[0][0], red[0][q]);
            red[1][0] = umax64(red[1][0], red[1][q]);
            red[2][0] = umax64(red[2][0], red[2][q]);
        }
        const double rmax = __longlong_as_double((long long)red[0][0]);
        const double xmax = __longlong_as_double((long long)red[1][0]);
        const double bmax = __longlong_as_double((long long)red[2][0]);
        const double knorm = __longlong_as_double((long long)stat[inst].knorm_bits);
        const double den = knorm * xmax + bmax;
        omega[inst] = den > 0.0 ? rmax / den : (den == 0.0 ? rmax : den);   // NaN stays NaN
    }
}

cudaError_t launch_resid_omega(const DevSched& s, const double* kvals, int64_t bs_slot, const double* x,
                               const double* b, double* r, double* part, const DevStat* stat, double* omega,
                               int batch, cudaStream_t st)
{
    const int nblk = sell_blocks(s);
    unsigned long long* up = reinterpret_cast<unsigned long long*>(part);
    resid_omega_part_kernel<<<dim3(nblk, batch), 256, 0, st>>>(s, kvals, bs_slot, x, b, r, up);
    omega_final_batched_kernel<<<batch, 256, 0, st>>>(nblk, up, stat, omega);
    return cudaGetLastError();
}

// explicit instantiations
#define KKT_INST(T)                                                                                              \
    template cudaError_t launch_scale<T>(const DevSched&, const DevNum<T>&, const double*, int, cudaStream_t);   \
    template cudaError_t launch_fronts_warp<T>(const DevSched&, const DevNum<T>&, const int*, int, int, int, int, \
                                               int, int, cudaStream_t);                                          \
    template cudaError_t launch_fronts_leaf<T>(const DevSched&, const DevNum<T>&, const int*, int, int, int,     \
                                               int, cudaStream_t);                                               \
    template cudaError_t launch_solve_bwd_leaf<T>(const DevSched&, const DevNum<T>&, const int*, int, int, int,  \
                                                  cudaStream_t);                                                 \
    template cudaError_t launch_fronts_cta<T>(const DevSched&, const DevNum<T>&, const int*, int, int, int,      \
                                              cudaStream_t);                                                     \
    template cudaError_t launch_fronts_panel<T>(const DevSched&, const DevNum<T>&, const int*, int, size_t, T*,  \
                                                int64_t, int, cudaStream_t);                                     \
    template cudaError_t launch_schur_tiles<T>(const DevSched&, const DevNum<T>&, const FrontTile*, int, int,    \
                                               int, cudaStream_t);                                               \
    template cudaError_t launch_solve_pre<T>(const DevSched&, const DevNum<T>&, const double*, int, cudaStream_t); \
    template cudaError_t launch_solve_post<T>(const DevSched&, const DevNum<T>&, double*, int, cudaStream_t);    \
    template cudaError_t launch_solve_fwd<T>(const DevSched&, const DevNum<T>&, const int*, int, int, int, int,  \
                                             cudaStream_t);                                                      \
    template cudaError_t launch_solve_bwd<T>(const DevSched&, const DevNum<T>&, const int*, int, int, int, int,  \
                                             cudaStream_t);                                                      \
    template cudaError_t launch_solve_fwd_cta<T>(const DevSched&, const DevNum<T>&, const int*, int, int, int,   \
                                                 int, cudaStream_t);                                             \
    template cudaError_t launch_solve_bwd_cta<T>(const DevSched&, const DevNum<T>&, const int*, int, int, int,   \
                                                 int, cudaStream_t);
KKT_INST(double)
KKT_INST(float)

// Raise each kernel's dynamic shared-memory limit to the device's opt-in
// maximum minus the kernel's static shared memory (once per process).
template <typename K>
static cudaError_t allow_smem(K kernel, int optin)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

cudaError_t configure_kernels()
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
    if ((e = allow_smem(front_warp_kernel<double>, optin))) return e;
    if ((e = allow_smem(front_warp_kernel<float>, optin))) return e;
    if ((e = allow_smem(front_cta_kernel<double>, optin))) return e;
    if ((e = allow_smem(front_cta_kernel<float>, optin))) return e;
    if ((e = allow_smem(front_panel_kernel<double>, optin))) return e;
    if ((e = allow_smem(front_panel_kernel<float>, optin))) return e;
    if ((e = allow_smem(solve_fwd_kernel<double>, optin))) return e;
    if ((e = allow_smem(solve_fwd_kernel<float>, optin))) return e;
    if ((e = allow_smem(solve_bwd_kernel<double>, optin))) return e;
    if ((e = allow_smem(solve_bwd_kernel<float>, optin))) return e;
    if ((e = allow_smem(solve_fwd_cta_kernel<double>, optin))) return e;
    if ((e = allow_smem(solve_fwd_cta_kernel<float>, optin))) return e;
    if ((e = allow_smem(solve_bwd_cta_kernel<double>, optin))) return e;
    if ((e = allow_smem(solve_bwd_cta_kernel<float>, optin))) return e;
    if ((e = allow_smem(schur_tile_kernel<double>, optin))) return e;
    if ((e = allow_smem(schur_tile_kernel<float>, optin))) return e;
    return configure_tree_kernels(optin);
}

}  // namespace kktgb
