// Approximate triangular solves by Jacobi sweeps, as the preconditioner of
// the refinement (Sec. V: the paper proposes iterative, Jacobi-type
// triangular solves instead of the level-scheduled exact ones, after Anzt et
// al.). With L unit lower and U upper, from y_0 = x_0 = 0:
//   y_{s+1} = c - (L - I) y_s
//   x_{s+1} = diag(U)^{-1} (y - (U - diag(U)) x_s)
// Each sweep is a product with the strict triangle, every row independent:
// no level schedule, no dependency between fronts within a launch. After s
// sweeps the result is exact on every unknown whose dependency chain in the
// factor is shorter than s; FGMRES (flexible: the preconditioner may change
// between iterations) corrects the rest.
//
// The factors stay in the multifrontal panels. A row i of L holds the
// strictly lower entries of its own front's pivot block and, for every
// descendant front whose contribution rows include i, that front's L21 row;
// kernel jacobi_l_part forms each front's L21 y_old (one value per
// contribution row, stored at the front's contribution-vector offsets) and
// jacobi_l_row gathers them per row in a fixed order (host-built row lists).
// A row of U lies entirely in its own front (U11 row and U12 row).
// The block variant (KKT_PRECOND_BLOCK_JACOBI) takes each front's pivots as
// a block solved exactly inside the sweep (Gauss-Seidel within the block):
//   y_{s+1} = L_D^{-1} (c - L_O y_s),   x_{s+1} = U_D^{-1} (y - U_O x_s)
// with L_D, U_D the fronts' pivot blocks and L_O, U_O the rest.
#include "kernels.cuh"

namespace kktgb {

namespace {

// t[rel_ptr[f] + r] = sum_p L21[r, p] y[first_f + p], one warp per front
template <typename T>
__global__ void __launch_bounds__(128) jacobi_l_part_kernel(DevSched s, DevNum<T> nm, const T* __restrict__ y,
                                                            T* __restrict__ t)
{
    const int f = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (f >= s.ns) return;
    const int first = s.sn_first[f], w = s.sn_first[f + 1] - first, F = s.sn_front[f], m = F - w;
    const T* pan = nm.panel + s.panel_off[f];
    T* out = t + s.rel_ptr[f];
    for (int r = lane; r < m; r += 32) {
        T acc = T(0);
        for (int p = 0; p < w; ++p) acc += pan[(w + r) + (int64_t)p * F] * y[first + p];
        out[r] = acc;
    }
}

// y_new[i] = c[i] - (own pivot block, strictly lower) - (descendants' parts)
template <typename T>
__global__ void __launch_bounds__(128) jacobi_l_row_kernel(DevSched s, DevNum<T> nm, const T* __restrict__ c,
                                                           const T* __restrict__ y, const T* __restrict__ t,
                                                           const int* __restrict__ lptr, const int* __restrict__ lidx,
                                                           T* __restrict__ ynew)
{
    const int f = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (f >= s.ns) return;
    const int first = s.sn_first[f], w = s.sn_first[f + 1] - first, F = s.sn_front[f];
    const T* pan = nm.panel + s.panel_off[f];
    for (int a = lane; a < w; a += 32) {
        const int i = first + a;
        T acc = c[i];
        for (int p = 0; p < a; ++p) acc -= pan[a + (int64_t)p * F] * y[first + p];
        for (int k = lptr[i]; k < lptr[i + 1]; ++k) acc -= t[lidx[k]];
        ynew[i] = acc;
    }
}

// x_new[i] = (y[i] - (U11 row, strictly upper) - (U12 row)) * (1 / u_ii)
template <typename T>
__global__ void __launch_bounds__(128) jacobi_u_kernel(DevSched s, DevNum<T> nm, const T* __restrict__ y,
                                                       const T* __restrict__ x, T* __restrict__ xnew)
{
    const int f = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (f >= s.ns) return;
    const int first = s.sn_first[f], w = s.sn_first[f + 1] - first, F = s.sn_front[f], m = F - w;
    const T* pan = nm.panel + s.panel_off[f];
    const T* U12 = pan + (int64_t)F * w;
    const int* R = s.rows + s.rows_ptr[f];
    for (int a = lane; a < w; a += 32) {
        T acc = y[first + a];
        for (int cc = a + 1; cc < w; ++cc) acc -= pan[a + (int64_t)cc * F] * x[first + cc];
        for (int tt = 0; tt < m; ++tt) acc -= U12[a + (int64_t)tt * w] * x[R[w + tt]];
        xnew[first + a] = acc * pivot_rcp(pan[a + (int64_t)a * F]);
    }
}

// Block variant (Gauss-Seidel inside each front): the pivots of a front
// form a block, solved exactly within the sweep from the other blocks'
// previous values. L: y_new[f] = L11^{-1} (c_f - descendants' parts), the
// unit lower pivot block substituted in pivot order; U: x_new[f] = U11^{-1}
// (y_f - U12 x_old), substituted backward with x_p = v_p * (1 / u_pp). One
// warp per front, the front's values in shared memory (w <= 64).
template <typename T>
__global__ void __launch_bounds__(128) jacobi_lb_kernel(DevSched s, DevNum<T> nm, const T* __restrict__ c,
                                                        const T* __restrict__ t, const int* __restrict__ lptr,
                                                        const int* __restrict__ lidx, T* __restrict__ ynew)
{
    __shared__ T vs[4][64];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int f = blockIdx.x * 4 + wid;
    if (f >= s.ns) return;
    const int first = s.sn_first[f], w = s.sn_first[f + 1] - first, F = s.sn_front[f];
    const T* pan = nm.panel + s.panel_off[f];
    T* v = vs[wid];
    for (int a = lane; a < w; a += 32) {
        const int i = first + a;
        T acc = c[i];
        for (int k = lptr[i]; k < lptr[i + 1]; ++k) acc -= t[lidx[k]];
        v[a] = acc;
    }
    __syncwarp();
    for (int p = 0; p < w; ++p) {
        const T xp = v[p];
        for (int a = p + 1 + lane; a < w; a += 32) v[a] -= pan[a + (int64_t)p * F] * xp;
        __syncwarp();
    }
    for (int a = lane; a < w; a += 32) ynew[first + a] = v[a];
}

template <typename T>
__global__ void __launch_bounds__(128) jacobi_ub_kernel(DevSched s, DevNum<T> nm, const T* __restrict__ y,
                                                        const T* __restrict__ x, T* __restrict__ xnew)
{
    __shared__ T vs[4][64];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int f = blockIdx.x * 4 + wid;
    if (f >= s.ns) return;
    const int first = s.sn_first[f], w = s.sn_first[f + 1] - first, F = s.sn_front[f], m = F - w;
    const T* pan = nm.panel + s.panel_off[f];
    const T* U12 = pan + (int64_t)F * w;
    const int* R = s.rows + s.rows_ptr[f];
    T* v = vs[wid];
    for (int a = lane; a < w; a += 32) {
        T acc = y[first + a];
        for (int tt = 0; tt < m; ++tt) acc -= U12[a + (int64_t)tt * w] * x[R[w + tt]];
        v[a] = acc;
    }
    __syncwarp();
    for (int p = w - 1; p >= 0; --p) {
        const T xp = v[p] * pivot_rcp(pan[p + (int64_t)p * F]);
        __syncwarp();
        if (lane == 0) v[p] = xp;
        for (int a = lane; a < p; a += 32) v[a] -= pan[a + (int64_t)p * F] * xp;
        __syncwarp();
    }
    for (int a = lane; a < w; a += 32) xnew[first + a] = v[a];
}

template <typename T>
__global__ void zero_kernel(int n, T* __restrict__ a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = T(0);
}

}  // namespace

// One application of the Jacobi preconditioner to the step-space vector in
// nm.vec (already permuted and scaled): `sweeps` sweeps with L, then with U;
// the result is left in nm.vec. Work buffers: ya, yb, xa (n each), t (one
// value per contribution row). Launches: 1 + 2 sweeps (L) + 1 + sweeps (U).
template <typename T>
cudaError_t launch_jacobi(const DevSched& s, const DevNum<T>& nm, int sweeps, bool block, const int* lptr,
                          const int* lidx, T* ya, T* yb, T* xa, T* t, int* launches, cudaStream_t st)
{
    const int n = s.n, blocks = (s.ns + 3) / 4, zb = (n + 255) / 256;
    const T* c = nm.vec;
    int k = 0;
    // L: y_0 = 0, y_1 = c, ...
    zero_kernel<T><<<zb, 256, 0, st>>>(n, ya);
    ++k;
    T* yo = ya;
    T* yn = yb;
    for (int sw = 0; sw < sweeps; ++sw) {
        jacobi_l_part_kernel<T><<<blocks, 128, 0, st>>>(s, nm, yo, t);
        if (block)
            jacobi_lb_kernel<T><<<blocks, 128, 0, st>>>(s, nm, c, t, lptr, lidx, yn);
        else
            jacobi_l_row_kernel<T><<<blocks, 128, 0, st>>>(s, nm, c, yo, t, lptr, lidx, yn);
        k += 2;
        T* tmp = yo;
        yo = yn;
        yn = tmp;
    }
    // U: x_0 = 0 in the free buffer A; sweeps alternate between B and A, and
    // the last one writes nm.vec (c, no longer needed)
    T* A = yn;
    T* Bf = xa;
    zero_kernel<T><<<zb, 256, 0, st>>>(n, A);
    ++k;
    const T* xo = A;
    for (int sw = 1; sw <= sweeps; ++sw) {
        T* dst = sw == sweeps ? nm.vec : ((sw % 2) ? Bf : A);
        if (block)
            jacobi_ub_kernel<T><<<blocks, 128, 0, st>>>(s, nm, yo, xo, dst);
        else
            jacobi_u_kernel<T><<<blocks, 128, 0, st>>>(s, nm, yo, xo, dst);
        ++k;
        xo = dst;
    }
    if (launches) *launches = k;
    return cudaGetLastError();
}

template cudaError_t launch_jacobi<double>(const DevSched&, const DevNum<double>&, int, bool, const int*, const int*,
                                           double*, double*, double*, double*, int*, cudaStream_t);
template cudaError_t launch_jacobi<float>(const DevSched&, const DevNum<float>&, int, bool, const int*, const int*,
                                          float*, float*, float*, float*, int*, cudaStream_t);

}  // namespace kktgb
