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
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* a, double v)
{
    atomicMax(a, (unsigned long long)__double_as_longlong(v));
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

template <typename T>
__device__ __forceinline__ T static_pivot(T piv, double floor_, DevStat* stat, bool count)
{
    double a = fabs((double)piv);
    if (!(a < 1e308)) {                       // NaN or Inf
        if (count) atomicExch(&stat->numeric_bad, 1);
        return piv;
    }
    if (a < floor_) {
        if (count) atomicAdd(&stat->n_perturbed, 1);
        return (T)(piv < T(0) ? -floor_ : floor_);
    }
    return piv;
}

// ------------------------------------------------------------------ Ruiz

__global__ void fill_kernel(int n, double* a, double v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// One Ruiz iteration, one warp per row: r_i = max_j |d_i k_ij d_j|,
// d_i <- d_i 2^round(-log2(r_i)/2). An iteration after one that changed
// nothing only copies d (the fixed point is reached).
__global__ void ruiz_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                            const double* __restrict__ v, const double* __restrict__ din,
                            double* __restrict__ dout, const int* changed_prev, int* changed_cur)
{
    int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    double di = din[row];
    if (changed_prev && *changed_prev == 0) {
        if (lane == 0) dout[row] = di;
        return;
    }
    double m = 0.0;
    for (int p = rp[row] + lane; p < rp[row + 1]; p += 32) m = fmax(m, fabs(di * v[p] * din[ci[p]]));
    m = warp_max(m);
    if (lane == 0) {
        double f = m > 0.0 ? pow2_inv_sqrt(m) : 1.0;
        dout[row] = di * f;
        if (f != 1.0) *changed_cur = 1;
    }
}

// D K D in factor precision, a copy of K for the residuals, max |D K D|
// (static-pivot reference) and ||K||_inf.
template <typename T>
__global__ void scale_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                             const double* __restrict__ v, const double* __restrict__ d,
                             T* __restrict__ sv, double* __restrict__ kcopy, DevStat* stat)
{
    int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    double amax = 0.0, rsum = 0.0;
    if (row < n) {
        double di = d[row];
        for (int p = rp[row] + lane; p < rp[row + 1]; p += 32) {
            const double k = v[p];
            double a = di * k * d[ci[p]];
            sv[p] = (T)a;
            kcopy[p] = k;
            amax = fmax(amax, fabs(a));
            rsum += fabs(k);
        }
    }
    amax = warp_max(amax);
    rsum = warp_sum(rsum);
    if (lane == 0 && row < n) {
        atomic_max_nonneg(&stat->amax_bits, amax);
        atomic_max_nonneg(&stat->knorm_bits, rsum);
    }
}

// ---------------------------------------------------------- front kernels

// Fronts with F <= 32: one warp per front, the whole front in shared memory,
// lane i owns row i of the front.
template <typename T>
__global__ void __launch_bounds__(128) front_warp_kernel(DevSched s, DevNum<T> nm, const int* __restrict__ fronts,
                                                         int count)
{
    __shared__ T sm[4][kWarpFrontMax * kWarpFrontMax];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int fi = blockIdx.x * 4 + wid;
    if (fi >= count) return;
    const int f = fronts[fi];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    T* Fm = sm[wid];
    for (int t = lane; t < F * F; t += 32) Fm[t] = T(0);
    __syncwarp();
    for (int64_t e = s.asm_ptr[f] + lane; e < s.asm_ptr[f + 1]; e += 32) Fm[s.asm_pos[e]] = nm.sv[s.asm_src[e]];
    __syncwarp();
    for (int c = s.child_ptr[f]; c < s.child_ptr[f + 1]; ++c) {
        const int ch = s.child_list[c];
        const int mc = s.sn_front[ch] - (s.sn_first[ch + 1] - s.sn_first[ch]);
        const T* cb = nm.cb + s.cb_off[ch];
        const int* rl = s.rel + s.rel_ptr[ch];
        for (int t = lane; t < mc * mc; t += 32) {
            int a = t % mc, b = t / mc;
            Fm[rl[a] + rl[b] * F] += cb[t];
        }
        __syncwarp();
    }
    const double floor_ = nm.pivot_eps * __longlong_as_double((long long)nm.stat->amax_bits);
    for (int p = 0; p < w; ++p) {
        const T pv = static_pivot(Fm[p + p * F], floor_, nm.stat, lane == 0);
        __syncwarp();
        if (lane == 0) Fm[p + p * F] = pv;
        const int i = lane;
        if (i > p && i < F) {
            const T l = Fm[i + p * F] / pv;
            Fm[i + p * F] = l;
            for (int j = p + 1; j < F; ++j) Fm[i + j * F] -= l * Fm[p + j * F];
        }
        __syncwarp();
    }
    T* pan = nm.panel + s.panel_off[f];
    const int m = F - w;
    for (int t = lane; t < F * w; t += 32) pan[t] = Fm[t];
    for (int t = lane; t < w * m; t += 32) {
        int a = t / m, b = t % m;
        pan[F * w + t] = Fm[a + (w + b) * F];
    }
    T* cbo = nm.cb + s.cb_off[f];
    for (int t = lane; t < m * m; t += 32) {
        int a = t % m, b = t / m;
        cbo[t] = Fm[(w + a) + (w + b) * F];
    }
}

// Fronts with F > 32 and a small contribution block: one CTA per front, the
// whole front in shared memory, right-looking rank-1 updates.
template <typename T>
__global__ void __launch_bounds__(256) front_cta_kernel(DevSched s, DevNum<T> nm, const int* __restrict__ fronts,
                                                        int count)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Fm = reinterpret_cast<T*>(smraw);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int f = fronts[blockIdx.x];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    for (int t = tid; t < F * F; t += nt) Fm[t] = T(0);
    __syncthreads();
    for (int64_t e = s.asm_ptr[f] + tid; e < s.asm_ptr[f + 1]; e += nt) Fm[s.asm_pos[e]] = nm.sv[s.asm_src[e]];
    __syncthreads();
    for (int c = s.child_ptr[f]; c < s.child_ptr[f + 1]; ++c) {
        const int ch = s.child_list[c];
        const int mc = s.sn_front[ch] - (s.sn_first[ch + 1] - s.sn_first[ch]);
        const T* cb = nm.cb + s.cb_off[ch];
        const int* rl = s.rel + s.rel_ptr[ch];
        for (int t = tid; t < mc * mc; t += nt) {
            int a = t % mc, b = t / mc;
            Fm[rl[a] + rl[b] * F] += cb[t];
        }
        __syncthreads();
    }
    const double floor_ = nm.pivot_eps * __longlong_as_double((long long)nm.stat->amax_bits);
    for (int p = 0; p < w; ++p) {
        const T pv = static_pivot(Fm[p + p * F], floor_, nm.stat, tid == 0);
        __syncthreads();
        if (tid == 0) Fm[p + p * F] = pv;
        for (int i = p + 1 + tid; i < F; i += nt) Fm[i + p * F] /= pv;
        __syncthreads();
        const int m = F - p - 1;
        for (int t = tid; t < m * m; t += nt) {
            const int i = p + 1 + t % m, j = p + 1 + t / m;
            Fm[i + j * F] -= Fm[i + p * F] * Fm[p + j * F];
        }
        __syncthreads();
    }
    T* pan = nm.panel + s.panel_off[f];
    const int m = F - w;
    for (int t = tid; t < F * w; t += nt) pan[t] = Fm[t];
    for (int t = tid; t < w * m; t += nt) {
        int a = t / m, b = t % m;
        pan[F * w + t] = Fm[a + (w + b) * F];
    }
    T* cbo = nm.cb + s.cb_off[f];
    for (int t = tid; t < m * m; t += nt) {
        int a = t % m, b = t / m;
        cbo[t] = Fm[(w + a) + (w + b) * F];
    }
}

// Fronts with a large contribution block: one CTA assembles the front (pivot
// columns and rows in shared memory, the (2,2) block directly in the front's
// contribution-block buffer) and factors the pivot panel; the Schur update of
// the (2,2) block is left to schur_tile_kernel, spread over many CTAs.
template <typename T>
__device__ __forceinline__ T* route(T* col, T* row, T* C, int F, int w, int a, int b)
{
    if (b < w) return col + a + (int64_t)b * F;
    if (a < w) return row + a + (int64_t)(b - w) * w;
    return C + (a - w) + (int64_t)(b - w) * (F - w);
}

template <typename T>
__global__ void __launch_bounds__(256) front_panel_kernel(DevSched s, DevNum<T> nm, const int* __restrict__ fronts,
                                                          int count, T* gscratch, int64_t sstride)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int f = fronts[blockIdx.x];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    const int m = F - w;
    T* col = gscratch ? gscratch + (int64_t)blockIdx.x * sstride : reinterpret_cast<T*>(smraw);
    T* row = col + (int64_t)F * w;
    T* C = nm.cb + s.cb_off[f];
    for (int64_t t = tid; t < (int64_t)F * w + (int64_t)w * m; t += nt) col[t] = T(0);
    for (int64_t t = tid; t < (int64_t)m * m; t += nt) C[t] = T(0);
    __syncthreads();
    for (int64_t e = s.asm_ptr[f] + tid; e < s.asm_ptr[f + 1]; e += nt) {
        const int pos = s.asm_pos[e];
        *route(col, row, C, F, w, pos % F, pos / F) = nm.sv[s.asm_src[e]];
    }
    __syncthreads();
    for (int c = s.child_ptr[f]; c < s.child_ptr[f + 1]; ++c) {
        const int ch = s.child_list[c];
        const int mc = s.sn_front[ch] - (s.sn_first[ch + 1] - s.sn_first[ch]);
        const T* cb = nm.cb + s.cb_off[ch];
        const int* rl = s.rel + s.rel_ptr[ch];
        for (int t = tid; t < mc * mc; t += nt) {
            int a = rl[t % mc], b = rl[t / mc];
            *route(col, row, C, F, w, a, b) += cb[t];
        }
        __syncthreads();
    }
    const double floor_ = nm.pivot_eps * __longlong_as_double((long long)nm.stat->amax_bits);
    for (int p = 0; p < w; ++p) {
        const T pv = static_pivot(col[p + (int64_t)p * F], floor_, nm.stat, tid == 0);
        __syncthreads();
        if (tid == 0) col[p + (int64_t)p * F] = pv;
        for (int i = p + 1 + tid; i < F; i += nt) col[i + (int64_t)p * F] /= pv;
        __syncthreads();
        const int mr = F - p - 1, mcn = w - p - 1;
        for (int t = tid; t < mr * mcn; t += nt) {
            const int i = p + 1 + t % mr, j = p + 1 + t / mr;
            col[i + (int64_t)j * F] -= col[i + (int64_t)p * F] * col[p + (int64_t)j * F];
        }
        const int ri = w - p - 1;
        for (int t = tid; t < ri * m; t += nt) {
            const int i = p + 1 + t % ri, j = t / ri;
            row[i + (int64_t)j * w] -= col[i + (int64_t)p * F] * row[p + (int64_t)j * w];
        }
        __syncthreads();
    }
    T* pan = nm.panel + s.panel_off[f];
    for (int64_t t = tid; t < (int64_t)F * w; t += nt) pan[t] = col[t];
    for (int64_t t = tid; t < (int64_t)w * m; t += nt) {
        int a = (int)(t / m), b = (int)(t % m);
        pan[(int64_t)F * w + t] = row[a + (int64_t)b * w];
    }
}

// C <- C - L21 U12 for one kTile x kTile tile of a panel-class front. The
// terms are applied in pivot order, one fused multiply-add each, exactly as
// the single-CTA kernels do.
template <typename T>
__global__ void __launch_bounds__(256) schur_tile_kernel(DevSched s, DevNum<T> nm, const FrontTile* __restrict__ tiles,
                                                         int count)
{
    constexpr int KB = 32;
    __shared__ T Ls[KB][kTile + 1];
    __shared__ T Us[KB][kTile + 1];
    const FrontTile tl = tiles[blockIdx.x];
    const int f = tl.front;
    const int w = s.sn_first[f + 1] - s.sn_first[f];
    const int F = s.sn_front[f];
    const int m = F - w;
    const int i0 = tl.ti * kTile, j0 = tl.tj * kTile;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;       // 8 warps
    const T* pan = nm.panel + s.panel_off[f];
    const T* L21 = pan + w;                                        // row r, col p at L21[r + p*F]
    const T* U12 = pan + (int64_t)F * w;                           // row p, col c at U12[p*m + c]
    T* C = nm.cb + s.cb_off[f];
    const int i = i0 + tx;
    T acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int j = j0 + ty + 8 * k;
        acc[k] = (i < m && j < m) ? C[i + (int64_t)j * m] : T(0);
    }
    for (int p0 = 0; p0 < w; p0 += KB) {
        const int kb = min(KB, w - p0);
        for (int t = threadIdx.x; t < KB * kTile; t += 256) {
            const int c = t / kTile, r = t % kTile;
            Ls[c][r] = (c < kb && i0 + r < m) ? L21[(i0 + r) + (int64_t)(p0 + c) * F] : T(0);
            Us[c][r] = (c < kb && j0 + r < m) ? U12[(int64_t)(p0 + c) * m + (j0 + r)] : T(0);
        }
        __syncthreads();
        for (int c = 0; c < kb; ++c) {
            const T l = Ls[c][tx];
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] -= l * Us[c][ty + 8 * k];
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int j = j0 + ty + 8 * k;
        if (i < m && j < m) C[i + (int64_t)j * m] = acc[k];
    }
}

// ------------------------------------------------------------ solve kernels

template <typename T>
__global__ void solve_pre_kernel(int n, const int* __restrict__ perm, const double* __restrict__ d,
                                 const double* __restrict__ b, T* __restrict__ vec)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        int o = perm[k];
        vec[k] = (T)(d[o] * b[o]);
    }
}

template <typename T>
__global__ void solve_post_kernel(int n, const int* __restrict__ perm, const double* __restrict__ d,
                                  const T* __restrict__ vec, double* __restrict__ x)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        int o = perm[k];
        x[o] = d[o] * (double)vec[k];
    }
}

// Forward substitution y = L^{-1} c, multifrontally: one warp per front
// gathers its pivot entries and its children's contribution vectors,
// eliminates its pivots, and leaves the updates of its non-pivot rows as its
// own contribution vector.
template <typename T>
__global__ void __launch_bounds__(128) solve_fwd_kernel(DevSched s, DevNum<T> nm, const int* __restrict__ fronts,
                                                        int count, int max_front)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int fi = blockIdx.x * 4 + wid;
    if (fi >= count) return;
    T* v = reinterpret_cast<T*>(smraw) + (int64_t)wid * max_front;
    const int f = fronts[fi];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    for (int a = lane; a < F; a += 32) v[a] = a < w ? nm.vec[first + a] : T(0);
    __syncwarp();
    for (int c = s.child_ptr[f]; c < s.child_ptr[f + 1]; ++c) {
        const int ch = s.child_list[c];
        const int mc = s.sn_front[ch] - (s.sn_first[ch + 1] - s.sn_first[ch]);
        const T* cv = nm.cbv + s.rel_ptr[ch];
        const int* rl = s.rel + s.rel_ptr[ch];
        for (int t = lane; t < mc; t += 32) v[rl[t]] += cv[t];
        __syncwarp();
    }
    const T* pan = nm.panel + s.panel_off[f];
    for (int p = 0; p < w; ++p) {
        const T xp = v[p];
        for (int i = p + 1 + lane; i < F; i += 32) v[i] -= pan[i + (int64_t)p * F] * xp;
        __syncwarp();
    }
    for (int a = lane; a < w; a += 32) nm.vec[first + a] = v[a];
    T* cv = nm.cbv + s.rel_ptr[f];
    for (int t = lane; t < F - w; t += 32) cv[t] = v[w + t];
}

// Back substitution x = U^{-1} y, top-down: one warp per front gathers the
// already-known solution entries of its non-pivot rows, subtracts U12 x, and
// back-substitutes with U11.
template <typename T>
__global__ void __launch_bounds__(128) solve_bwd_kernel(DevSched s, DevNum<T> nm, const int* __restrict__ fronts,
                                                        int count, int max_front)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int fi = blockIdx.x * 4 + wid;
    if (fi >= count) return;
    T* v = reinterpret_cast<T*>(smraw) + (int64_t)wid * max_front;    // v[0..w): t, v[w..F): x of the other rows
    const int f = fronts[fi];
    const int first = s.sn_first[f];
    const int w = s.sn_first[f + 1] - first;
    const int F = s.sn_front[f];
    const int m = F - w;
    const int* R = s.rows + s.rows_ptr[f];
    for (int t = lane; t < m; t += 32) v[w + t] = nm.vec[R[w + t]];
    __syncwarp();
    const T* pan = nm.panel + s.panel_off[f];
    const T* U12 = pan + (int64_t)F * w;
    for (int a = 0; a < w; ++a) {
        T acc = T(0);
        for (int t = lane; t < m; t += 32) acc += U12[(int64_t)a * m + t] * v[w + t];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) v[a] = nm.vec[first + a] - acc;
    }
    __syncwarp();
    for (int p = w - 1; p >= 0; --p) {
        const T xp = v[p] / pan[p + (int64_t)p * F];
        __syncwarp();
        if (lane == 0) v[p] = xp;
        for (int a = lane; a < p; a += 32) v[a] -= pan[a + (int64_t)p * F] * xp;
        __syncwarp();
    }
    for (int a = lane; a < w; a += 32) nm.vec[first + a] = v[a];
}

// ---------------------------------------------------------- FP64 vectors

__global__ void spmv_resid_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                  const double* __restrict__ v, const double* __restrict__ x,
                                  const double* __restrict__ b, double* __restrict__ r)
{
    int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0;
    for (int p = rp[row] + lane; p < rp[row + 1]; p += 32) s += v[p] * x[ci[p]];
    s = warp_sum(s);
    if (lane == 0) r[row] = b ? b[row] - s : s;
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

__global__ void norms_part_kernel(int n, const double* __restrict__ a, double* __restrict__ part)
{
    __shared__ double smax[32], ssum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double mx = 0.0, sq = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = a[i];
        mx = fmax(mx, fabs(v));
        sq += v * v;
    }
    mx = warp_max(mx);
    sq = warp_sum(sq);
    if (lane == 0) { smax[wid] = mx; ssum[wid] = sq; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double M = 0.0, S = 0.0;
        for (int q = 0; q < nw; ++q) { M = fmax(M, smax[q]); S += ssum[q]; }
        part[2 * blockIdx.x] = M;
        part[2 * blockIdx.x + 1] = S;
    }
}

__global__ void norms_final_kernel(int nblk, const double* __restrict__ part, double* __restrict__ out)
{
    double M = 0.0, S = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) { M = fmax(M, part[2 * b]); S += part[2 * b + 1]; }
    M = warp_max(M);
    S = warp_sum(S);
    if (threadIdx.x == 0) { out[0] = M; out[1] = S; }
}

}  // namespace

// ================================================================ launchers

static inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

cudaError_t launch_zero_stat(DevStat* stat, cudaStream_t st)
{
    return cudaMemsetAsync(stat, 0, sizeof(DevStat), st);
}

cudaError_t launch_ruiz(const DevSched& s, const double* vals, double* d, double* dtmp, int iters,
                        DevStat* stat, double** d_final, cudaStream_t st)
{
    fill_kernel<<<cdiv(s.n, 256), 256, 0, st>>>(s.n, d, 1.0);
    double* a = d;
    double* b = dtmp;
    for (int it = 0; it < iters; ++it) {
        ruiz_kernel<<<cdiv((int64_t)s.n * 32, 256), 256, 0, st>>>(
            s.n, s.rowptr, s.colidx, vals, a, b, it > 0 ? &stat->ruiz_changed[it - 1] : nullptr,
            &stat->ruiz_changed[it]);
        double* t = a; a = b; b = t;
    }
    *d_final = a;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale(const DevSched& s, const DevNum<T>& nm, const double* d, cudaStream_t st)
{
    scale_kernel<T><<<cdiv((int64_t)s.n * 32, 256), 256, 0, st>>>(s.n, s.rowptr, s.colidx, nm.vals, d, nm.sv,
                                                                   nm.kcopy, nm.stat);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fronts_warp(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    front_warp_kernel<T><<<cdiv(count, 4), 128, 0, st>>>(s, nm, fronts, count);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fronts_cta(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, int max_front,
                              cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    size_t smem = (size_t)max_front * max_front * sizeof(T);
    front_cta_kernel<T><<<count, 256, smem, st>>>(s, nm, fronts, count);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fronts_panel(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count,
                                size_t smem_bytes, T* gscratch, int64_t scratch_stride, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    front_panel_kernel<T><<<count, 256, gscratch ? 0 : smem_bytes, st>>>(s, nm, fronts, count, gscratch,
                                                                          scratch_stride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_schur_tiles(const DevSched& s, const DevNum<T>& nm, const FrontTile* tiles, int count,
                               cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    schur_tile_kernel<T><<<count, 256, 0, st>>>(s, nm, tiles, count);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_pre(const DevSched& s, const DevNum<T>& nm, const double* b, cudaStream_t st)
{
    solve_pre_kernel<T><<<cdiv(s.n, 256), 256, 0, st>>>(s.n, s.perm, nm.d, b, nm.vec);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_post(const DevSched& s, const DevNum<T>& nm, double* x, cudaStream_t st)
{
    solve_post_kernel<T><<<cdiv(s.n, 256), 256, 0, st>>>(s.n, s.perm, nm.d, nm.vec, x);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_fwd(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, int max_front,
                             cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    solve_fwd_kernel<T><<<cdiv(count, 4), 128, 4 * (size_t)max_front * sizeof(T), st>>>(s, nm, fronts, count,
                                                                                         max_front);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_bwd(const DevSched& s, const DevNum<T>& nm, const int* fronts, int count, int max_front,
                             cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    solve_bwd_kernel<T><<<cdiv(count, 4), 128, 4 * (size_t)max_front * sizeof(T), st>>>(s, nm, fronts, count,
                                                                                         max_front);
    return cudaGetLastError();
}

cudaError_t launch_spmv_resid(int n, const int* rp, const int* ci, const double* v, const double* x,
                              const double* b, double* r, cudaStream_t st)
{
    spmv_resid_kernel<<<cdiv((int64_t)n * 32, 256), 256, 0, st>>>(n, rp, ci, v, x, b, r);
    return cudaGetLastError();
}

cudaError_t launch_spmv(int n, const int* rp, const int* ci, const double* v, const double* x, double* y,
                        cudaStream_t st)
{
    spmv_resid_kernel<<<cdiv((int64_t)n * 32, 256), 256, 0, st>>>(n, rp, ci, v, x, nullptr, y);
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

cudaError_t launch_norms(int n, const double* a, double* out, cudaStream_t st)
{
    double* part = out + 2;
    norms_part_kernel<<<kRedBlocks, 256, 0, st>>>(n, a, part);
    norms_final_kernel<<<1, 32, 0, st>>>(kRedBlocks, part, out);
    return cudaGetLastError();
}

// explicit instantiations
#define KKT_INST(T)                                                                                              \
    template cudaError_t launch_scale<T>(const DevSched&, const DevNum<T>&, const double*, cudaStream_t);        \
    template cudaError_t launch_fronts_warp<T>(const DevSched&, const DevNum<T>&, const int*, int, cudaStream_t); \
    template cudaError_t launch_fronts_cta<T>(const DevSched&, const DevNum<T>&, const int*, int, int,           \
                                              cudaStream_t);                                                     \
    template cudaError_t launch_fronts_panel<T>(const DevSched&, const DevNum<T>&, const int*, int, size_t, T*,  \
                                                int64_t, cudaStream_t);                                          \
    template cudaError_t launch_schur_tiles<T>(const DevSched&, const DevNum<T>&, const FrontTile*, int,         \
                                               cudaStream_t);                                                    \
    template cudaError_t launch_solve_pre<T>(const DevSched&, const DevNum<T>&, const double*, cudaStream_t);    \
    template cudaError_t launch_solve_post<T>(const DevSched&, const DevNum<T>&, double*, cudaStream_t);         \
    template cudaError_t launch_solve_fwd<T>(const DevSched&, const DevNum<T>&, const int*, int, int,            \
                                             cudaStream_t);                                                      \
    template cudaError_t launch_solve_bwd<T>(const DevSched&, const DevNum<T>&, const int*, int, int,            \
                                             cudaStream_t);
KKT_INST(double)
KKT_INST(float)

// set dynamic shared-memory limits once per process
cudaError_t configure_kernels()
{
    cudaError_t e;
    const int lim = 227 * 1024;
    if ((e = cudaFuncSetAttribute(front_cta_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(front_cta_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(front_panel_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(front_panel_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(solve_fwd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(solve_fwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(solve_bwd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(solve_bwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    return cudaSuccess;
}

}  // namespace kktgb
