// The interior-point loop around the linear solver (Sec. II: Newton's method
// on the barrier problem with continuation mu -> 0, one KKT system K_k per
// iteration, Eq. 11), on the GPU: kkt_model_set_limits, kkt_ipm_solve.
//
// Problem: min sum c2 Pg^2 + rho theta_ref^2 subject to the power balance c_E(x) = 0, the line
// limits c_I(x) + s = u (|S|^2 at both ends, u = Smax^2, s >= 0) and bounds
// xL <= x <= xU on |V|, Pg, Qg (Eqs. 1-4, slacks as in Eqs. 5-7). The term
// rho theta_ref^2 fixes the reference angle without changing the optimal cost
// (everything else depends on angle differences only): it removes the
// uniform angle shift, a null direction of K otherwise held only by dw. Each
// iteration: evaluate the flows and constraints, assemble K (the model's
// kernels) with the barrier diagonal Sigma_x = zL/(x-xL) + zU/(xU-x) on the
// primal diagonal and the slack term s/w on the flow rows' (2,2) diagonal,
// read J^T lambda off K, measure the optimality error, update mu, form the
// right-hand side, refactor and refine (the library's path), recover the
// bound and slack steps, take the fraction-to-the-boundary step. Every vector
// step is a kernel; per iteration the host reads a few scalars (the error
// measures, then the two step lengths) to decide mu and alpha.
#include "../../include/kkt.h"
#include "model.hpp"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <type_traits>
#include <vector>

namespace {

constexpr int kIpmThreads = 256;
constexpr int kIpmBlocks = 304;                 // 2 x 152 SMs, grid-stride loops
constexpr int kIpmRed = 8;                      // reduced quantities per block

__device__ __forceinline__ unsigned long long mag(double v)
{
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long umax(unsigned long long a, unsigned long long b) { return a > b ? a : b; }
__device__ __forceinline__ unsigned long long umin(unsigned long long a, unsigned long long b) { return a < b ? a : b; }

// flows leaving each end of every line: PQ[4l..4l+3] = (Pf, Qf, Pt, Qt)
__global__ void ipm_flows_kernel(int nl, const int* __restrict__ lf, const int* __restrict__ lt,
                                 const double* __restrict__ lg, const double* __restrict__ lb,
                                 const double* __restrict__ V, const double* __restrict__ th, double* __restrict__ PQ)
{
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += gridDim.x * blockDim.x) {
        const int i = lf[l], j = lt[l];
        const double g = lg[l], b = lb[l];
        const double t = th[i] - th[j];
        const double c = cos(t), s = sin(t);
        for (int e = 0; e < 2; ++e) {
            const double Va = e ? V[j] : V[i], Vb = e ? V[i] : V[j];
            const double sa = e ? -s : s;
            const double A = g * c + b * sa, Bq = g * sa - b * c;
            PQ[4 * l + 2 * e] = g * Va * Va - Va * Vb * A;
            PQ[4 * l + 2 * e + 1] = -b * Va * Va - Va * Vb * Bq;
        }
    }
}

// c_E: per bus, generation - load - flows leaving (P rows, then Q rows);
// c_I: |S|^2 at the from ends, then at the to ends
__global__ void ipm_constraints_kernel(int nb, int nl, int flow, const int* __restrict__ bus_ptr,
                                       const int* __restrict__ bus_end, const int* __restrict__ gen_of_bus,
                                       const double* __restrict__ Pg, const double* __restrict__ Qg,
                                       const double* __restrict__ Pd, const double* __restrict__ Qd,
                                       const double* __restrict__ PQ, double* __restrict__ cE, double* __restrict__ cI)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
        const int k = gen_of_bus[i];
        double p = (k >= 0 ? Pg[k] : 0.0) - Pd[i];
        double q = (k >= 0 ? Qg[k] : 0.0) - Qd[i];
        for (int e = bus_ptr[i]; e < bus_ptr[i + 1]; ++e) {
            const int le = bus_end[e];
            p -= PQ[2 * le];
            q -= PQ[2 * le + 1];
        }
        cE[i] = p;
        cE[nb + i] = q;
    }
    if (flow)
        for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += gridDim.x * blockDim.x) {
            const double Pf = PQ[4 * l], Qf = PQ[4 * l + 1], Pt = PQ[4 * l + 2], Qt = PQ[4 * l + 3];
            cI[l] = Pf * Pf + Qf * Qf;
            cI[nl + l] = Pt * Pt + Qt * Qt;
        }
}

// Sigma_x and the slack term s/w of the flow rows (0 on the balance rows)
__global__ void ipm_diag_kernel(int np, int m, int mE, int iref, double pin2, const double* __restrict__ x,
                                const double* __restrict__ lo,
                                const double* __restrict__ hi, const double* __restrict__ zL,
                                const double* __restrict__ zU, const double* __restrict__ s,
                                const double* __restrict__ w, double* __restrict__ sigma, double* __restrict__ D)
{
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += stride) {
        double sg = 0.0;
        if (isfinite(lo[i])) sg += zL[i] / (x[i] - lo[i]);
        if (isfinite(hi[i])) sg += zU[i] / (hi[i] - x[i]);
        if (i == iref) sg += pin2;                                 // Hessian of the reference-angle term
        sigma[i] = sg;
    }
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += stride)
        D[r] = r < mE ? 0.0 : s[r - mE] / w[r - mE];
}

// J^T lambda: the primal rows of K times (0; lambda), i.e. the J^T block of the
// assembled K (its values do not depend on lambda, Sigma or the (2,2) block)
__global__ void ipm_jtlam_kernel(int np, const int* __restrict__ rp, const int* __restrict__ ci,
                                 const double* __restrict__ vals, const double* __restrict__ lam,
                                 double* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            const int c = ci[p];
            if (c >= np) acc += vals[p] * lam[c - np];
        }
        out[i] = acc;
    }
}

// Block reduction of kIpmRed quantities into red[blockIdx.x * kIpmRed + q]:
// maxima / minima on bit patterns of non-negative values (NaN sorts above
// +Inf), sums in FP64 in a fixed order.
__device__ void block_reduce(const unsigned long long (&mx)[kIpmRed], const bool (&is_min)[kIpmRed],
                             const bool (&is_sum)[kIpmRed], const double (&sm)[kIpmRed], double* red)
{
    __shared__ unsigned long long sb[kIpmRed][kIpmThreads / 32];
    __shared__ double ss[kIpmRed][kIpmThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < kIpmRed; ++q) {
        unsigned long long v = mx[q];
        double d = sm[q];
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
            v = is_min[q] ? umin(v, u) : umax(v, u);
            d += __shfl_xor_sync(0xffffffffu, d, o);
        }
        if (lane == 0) { sb[q][wid] = v; ss[q][wid] = d; }
    }
    __syncthreads();
    if (threadIdx.x < kIpmRed) {
        const int q = threadIdx.x;
        unsigned long long v = sb[q][0];
        double d = ss[q][0];
        for (int k = 1; k < kIpmThreads / 32; ++k) {
            v = is_min[q] ? umin(v, sb[q][k]) : umax(v, sb[q][k]);
            d += ss[q][k];
        }
        red[blockIdx.x * kIpmRed + q] = is_sum[q] ? d : __longlong_as_double((long long)v);
    }
}

// Optimality measures of the current iterate: [0] ||grad F + J^T lam - zL + zU||,
// [1] ||c_E||, [2] ||c_I + s - u||, [3] ||lam_I - w||, [4] largest and [5]
// smallest complementarity product, [6] the objective (sum), [7] unused.
__global__ void __launch_bounds__(kIpmThreads) ipm_errors_kernel(
    int np, int nb, int ng, int mI, int iref, double pin2, const double* __restrict__ x,
    const double* __restrict__ lo, const double* __restrict__ hi, const double* __restrict__ zL,
    const double* __restrict__ zU, const double* __restrict__ twoc2, const double* __restrict__ jtl,
    const double* __restrict__ cE,
    const double* __restrict__ cI, const double* __restrict__ s, const double* __restrict__ w,
    const double* __restrict__ u, const double* __restrict__ lamI, double* __restrict__ red)
{
    unsigned long long mx[kIpmRed] = {0, 0, 0, 0, 0, 0x7ff0000000000000ull, 0, 0};
    double sm[kIpmRed] = {0, 0, 0, 0, 0, 0, 0, 0};
    const bool is_min[kIpmRed] = {false, false, false, false, false, true, false, false};
    const bool is_sum[kIpmRed] = {false, false, false, false, false, false, true, false};
    const int stride = gridDim.x * blockDim.x, t0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int pg0 = 2 * nb;
    for (int i = t0; i < np; i += stride) {
        double grad = 0.0;
        if ((i >= pg0 && i < pg0 + ng) || i == iref) {
            grad = (i == iref ? pin2 : twoc2[i - pg0]) * x[i];
            sm[6] += 0.5 * grad * x[i];                               // c2 Pg^2, rho theta_ref^2
        }
        mx[0] = umax(mx[0], mag(grad + jtl[i] - zL[i] + zU[i]));
        if (isfinite(lo[i])) {
            const double p = (x[i] - lo[i]) * zL[i];
            mx[4] = umax(mx[4], mag(p));
            mx[5] = umin(mx[5], mag(p));
        }
        if (isfinite(hi[i])) {
            const double p = (hi[i] - x[i]) * zU[i];
            mx[4] = umax(mx[4], mag(p));
            mx[5] = umin(mx[5], mag(p));
        }
    }
    for (int r = t0; r < 2 * nb; r += stride) mx[1] = umax(mx[1], mag(cE[r]));
    for (int k = t0; k < mI; k += stride) {
        mx[2] = umax(mx[2], mag(cI[k] + s[k] - u[k]));
        mx[3] = umax(mx[3], mag(lamI[k] - w[k]));
        const double p = s[k] * w[k];
        mx[4] = umax(mx[4], mag(p));
        mx[5] = umin(mx[5], mag(p));
    }
    block_reduce(mx, is_min, is_sum, sm, red);
}

// right-hand side of the Newton system at barrier parameter mu
__global__ void ipm_rhs_kernel(int np, int nb, int ng, int mI, int iref, double pin2, double mu,
                               const double* __restrict__ x,
                               const double* __restrict__ lo, const double* __restrict__ hi,
                               const double* __restrict__ twoc2, const double* __restrict__ jtl,
                               const double* __restrict__ cE, const double* __restrict__ cI,
                               const double* __restrict__ s, const double* __restrict__ w,
                               const double* __restrict__ u, const double* __restrict__ lamI,
                               double* __restrict__ rhs)
{
    const int stride = gridDim.x * blockDim.x, t0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int pg0 = 2 * nb;
    for (int i = t0; i < np; i += stride) {
        double r = jtl[i];
        if (i >= pg0 && i < pg0 + ng) r += twoc2[i - pg0] * x[i];
        if (i == iref) r += pin2 * x[i];
        if (isfinite(lo[i])) r -= mu / (x[i] - lo[i]);
        if (isfinite(hi[i])) r += mu / (hi[i] - x[i]);
        rhs[i] = -r;
    }
    for (int r = t0; r < 2 * nb; r += stride) rhs[np + r] = -cE[r];
    for (int k = t0; k < mI; k += stride)
        rhs[np + 2 * nb + k] = -(cI[k] + s[k] - u[k]) - (mu / s[k] - lamI[k]) * (s[k] / w[k]);
}

// Bound and slack steps from the Newton direction, and the largest primal
// ([0]) and dual ([1]) step lengths that keep every distance above (1 - tau)
// times its value (minima of positive ratios, +Inf when nothing limits).
__global__ void __launch_bounds__(kIpmThreads) ipm_step_kernel(
    int np, int mI, int mE, double mu, double tau, const double* __restrict__ x, const double* __restrict__ lo,
    const double* __restrict__ hi, const double* __restrict__ zL, const double* __restrict__ zU,
    const double* __restrict__ s, const double* __restrict__ w, const double* __restrict__ lamI,
    const double* __restrict__ dir, double* __restrict__ dzL, double* __restrict__ dzU, double* __restrict__ ds,
    double* __restrict__ dw, double* __restrict__ red)
{
    const unsigned long long inf = 0x7ff0000000000000ull;
    unsigned long long mx[kIpmRed] = {inf, inf, 0, 0, 0, 0, 0, 0};
    double sm[kIpmRed] = {0, 0, 0, 0, 0, 0, 0, 0};
    const bool is_min[kIpmRed] = {true, true, false, false, false, false, false, false};
    const bool is_sum[kIpmRed] = {false, false, false, false, false, false, false, false};
    const int stride = gridDim.x * blockDim.x, t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = t0; i < np; i += stride) {
        const double dx = dir[i];
        double a = 0.0, b = 0.0;
        if (isfinite(lo[i])) {
            const double dl = x[i] - lo[i];
            a = mu / dl - zL[i] - (zL[i] / dl) * dx;
            if (dx < 0.0) mx[0] = umin(mx[0], mag(-tau * dl / dx));
            if (a < 0.0) mx[1] = umin(mx[1], mag(-tau * zL[i] / a));
        }
        if (isfinite(hi[i])) {
            const double du = hi[i] - x[i];
            b = mu / du - zU[i] + (zU[i] / du) * dx;
            if (dx > 0.0) mx[0] = umin(mx[0], mag(tau * du / dx));
            if (b < 0.0) mx[1] = umin(mx[1], mag(-tau * zU[i] / b));
        }
        dzL[i] = a;
        dzU[i] = b;
    }
    for (int k = t0; k < mI; k += stride) {
        const double dl = dir[np + mE + k];
        const double dsk = (mu / s[k] - lamI[k] - dl) * (s[k] / w[k]);
        const double dwk = mu / s[k] - w[k] - (w[k] / s[k]) * dsk;
        if (dsk < 0.0) mx[0] = umin(mx[0], mag(-tau * s[k] / dsk));
        if (dwk < 0.0) mx[1] = umin(mx[1], mag(-tau * w[k] / dwk));
        ds[k] = dsk;
        dw[k] = dwk;
    }
    block_reduce(mx, is_min, is_sum, sm, red);
}

__global__ void ipm_update_kernel(int np, int m, int mI, double ap, double ad, double* __restrict__ x,
                                  double* __restrict__ lam, double* __restrict__ s, double* __restrict__ w,
                                  double* __restrict__ zL, double* __restrict__ zU, const double* __restrict__ dir,
                                  const double* __restrict__ dzL, const double* __restrict__ dzU,
                                  const double* __restrict__ ds, const double* __restrict__ dw)
{
    const int stride = gridDim.x * blockDim.x, t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = t0; i < np; i += stride) {
        x[i] += ap * dir[i];
        zL[i] += ad * dzL[i];
        zU[i] += ad * dzU[i];
    }
    for (int r = t0; r < m; r += stride) lam[r] += ap * dir[np + r];
    for (int k = t0; k < mI; k += stride) {
        s[k] += ap * ds[k];
        w[k] += ad * dw[k];
    }
}

// Starting point: x pushed into the interior, s = max(u - c_I(x), push u),
// lambda = 0, zL = mu0/(x - xL), zU = mu0/(xU - x), w = mu0/s.
__global__ void ipm_push_kernel(int np, double push, const double* __restrict__ lo, const double* __restrict__ hi,
                                double* __restrict__ x)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        double v = x[i];
        const bool bl = isfinite(lo[i]), bu = isfinite(hi[i]);
        const double span = (bl && bu) ? hi[i] - lo[i] : 1.0;
        if (bl) v = fmax(v, lo[i] + push * span);
        if (bu) v = fmin(v, hi[i] - push * span);
        x[i] = v;
    }
}

__global__ void ipm_start_kernel(int np, int m, int mI, double mu0, double push, const double* __restrict__ x,
                                 const double* __restrict__ lo, const double* __restrict__ hi,
                                 const double* __restrict__ cI, const double* __restrict__ u,
                                 double* __restrict__ lam, double* __restrict__ s, double* __restrict__ w,
                                 double* __restrict__ zL, double* __restrict__ zU)
{
    const int stride = gridDim.x * blockDim.x, t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = t0; i < np; i += stride) {
        zL[i] = isfinite(lo[i]) ? mu0 / (x[i] - lo[i]) : 0.0;
        zU[i] = isfinite(hi[i]) ? mu0 / (hi[i] - x[i]) : 0.0;
    }
    for (int r = t0; r < m; r += stride) lam[r] = 0.0;
    for (int k = t0; k < mI; k += stride) {
        s[k] = fmax(u[k] - cI[k], push * u[k]);
        w[k] = mu0 / s[k];
    }
}

// the per-block results of block_reduce into out[0 .. kIpmRed)
__global__ void ipm_final_kernel(int nblk, const double* __restrict__ red, int min_mask, int sum_mask,
                                 double* __restrict__ out)
{
    const int q = threadIdx.x;
    if (q >= kIpmRed) return;
    const bool mn = (min_mask >> q) & 1, su = (sum_mask >> q) & 1;
    double d = 0.0;
    unsigned long long v = mn ? 0x7ff0000000000000ull : 0ull;
    for (int b = 0; b < nblk; ++b) {
        const double e = red[b * kIpmRed + q];
        if (su) d += e;
        else {
            const unsigned long long bits = mag(e);
            v = mn ? umin(v, bits) : umax(v, bits);
        }
    }
    out[q] = su ? d : __longlong_as_double((long long)v);
}

}  // namespace

extern "C" {

void kkt_ipm_default_options(kkt_ipm_options* o)
{
    if (!o) return;
    o->tol = 1e-7;
    o->max_iter = 200;
    o->mu0 = 0.1;
    o->kappa_eps = 10.0;
    o->kappa_mu = 0.2;
    o->theta_mu = 1.5;
    o->tau_min = 0.99;
    o->delta_w = 1e-8;
    o->delta_c = 1e-8;
    o->push = 1e-2;
    o->lin_tol = 1e-10;
    o->angle_ref = 0;
    o->angle_pin = 1.0;
}

kkt_status kkt_model_set_limits(kkt_model* m, const double* h_Pd, const double* h_Qd, const double* h_Vmin,
                                const double* h_Vmax, const double* h_Pmin, const double* h_Pmax,
                                const double* h_Qmin, const double* h_Qmax, const double* h_Smax)
{
    if (!m || !m->base) return m ? KKT_E_STATE : KKT_E_ARG;
    const int B = m->nb, L = m->nl, G = m->ng, np = m->n_primal, n = m->n;
    if (!h_Pd || !h_Qd || !h_Vmin || !h_Vmax || (G && (!h_Pmin || !h_Pmax || !h_Qmin || !h_Qmax)) ||
        (m->flow && L && !h_Smax))
        return KKT_E_ARG;
    for (int i = 0; i < B; ++i)
        if (!(h_Vmin[i] > 0.0 && h_Vmin[i] < h_Vmax[i]) || !std::isfinite(h_Vmax[i]) || !std::isfinite(h_Pd[i]) ||
            !std::isfinite(h_Qd[i]))
            return KKT_E_ARG;
    for (int k = 0; k < G; ++k)
        if (!(h_Pmin[k] < h_Pmax[k]) || !(h_Qmin[k] < h_Qmax[k]) || !std::isfinite(h_Pmin[k]) ||
            !std::isfinite(h_Pmax[k]) || !std::isfinite(h_Qmin[k]) || !std::isfinite(h_Qmax[k]))
            return KKT_E_ARG;
    if (m->flow)
        for (int l = 0; l < L; ++l)
            if (!(h_Smax[l] > 0.0) || !std::isfinite(h_Smax[l])) return KKT_E_ARG;
    const int mI = m->flow ? 2 * L : 0, md = n - np;
    std::vector<double> lo(np), hi(np), u(std::max(mI, 1), 0.0);
    std::vector<int> bus_ptr(B + 1, 0), bus_end(2 * (size_t)L), gen_of_bus(B, -1);
    try {
        for (int i = 0; i < B; ++i) {
            lo[i] = h_Vmin[i];
            hi[i] = h_Vmax[i];
            lo[B + i] = -INFINITY;
            hi[B + i] = INFINITY;
        }
        for (int k = 0; k < G; ++k) {
            lo[2 * B + k] = h_Pmin[k];
            hi[2 * B + k] = h_Pmax[k];
            lo[2 * B + G + k] = h_Qmin[k];
            hi[2 * B + G + k] = h_Qmax[k];
            gen_of_bus[m->gen_bus[k]] = k;
        }
        for (int l = 0; l < mI / 2; ++l) u[l] = u[L + l] = h_Smax[l] * h_Smax[l];
        for (int l = 0; l < L; ++l) { bus_ptr[m->from[l] + 1]++; bus_ptr[m->to[l] + 1]++; }
        for (int i = 0; i < B; ++i) bus_ptr[i + 1] += bus_ptr[i];
        std::vector<int> fill(bus_ptr.begin(), bus_ptr.end() - 1);
        for (int l = 0; l < L; ++l) {                    // line end index le = 2 l + end, in line order
            bus_end[fill[m->from[l]]++] = 2 * l;
            bus_end[fill[m->to[l]]++] = 2 * l + 1;
        }
    } catch (const std::bad_alloc&) {
        return KKT_E_NOMEM;
    }
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t nd = (size_t)np, ndu = (size_t)std::max(mI, 1), nm = (size_t)std::max(md, 1);
    const size_t sz[] = {al(8 * (size_t)B), al(8 * (size_t)B), al(8 * nd), al(8 * nd), al(8 * ndu),
                         al(4 * (size_t)(B + 1)), al(4 * std::max<size_t>(2 * (size_t)L, 1)), al(4 * (size_t)B),
                         al(4 * (size_t)(n + 1)), al(4 * (size_t)m->nnz),
                         al(8 * ndu), al(8 * ndu), al(8 * nd), al(8 * nd),                    // s w zL zU
                         al(8 * 4 * std::max<size_t>((size_t)L, 1)), al(8 * 2 * (size_t)B), al(8 * ndu),   // PQ cE cI
                         al(8 * nd), al(8 * nm), al(8 * (size_t)m->nnz), al(8 * nd),          // sigma D vals jtl
                         al(8 * (size_t)n), al(8 * (size_t)n), al(8 * nd), al(8 * nd),         // rhs dir dzL dzU
                         al(8 * ndu), al(8 * ndu), al(8 * (size_t)kIpmBlocks * kIpmRed + 64)}; // ds dw red
    size_t total = 0;
    for (size_t v : sz) total += v;
    if (m->ipm_base) { cudaFree(m->ipm_base); m->ipm_base = nullptr; }
    if (cudaMalloc(&m->ipm_base, total) != cudaSuccess) {
        cudaGetLastError();
        m->ipm_base = nullptr;
        return KKT_E_NOMEM;
    }
    if (!m->ipm_pin && cudaMallocHost(&m->ipm_pin, 8 * kIpmRed * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        m->ipm_pin = nullptr;
        return KKT_E_NOMEM;
    }
    char* p = m->ipm_base;
    size_t k = 0;
    auto take = [&](auto*& dst) { dst = reinterpret_cast<std::remove_reference_t<decltype(dst)>>(p); p += sz[k++]; };
    take(m->d_Pd); take(m->d_Qd); take(m->d_lo); take(m->d_hi); take(m->d_u);
    take(m->d_bus_ptr); take(m->d_bus_end); take(m->d_gen_of_bus); take(m->d_rowptr); take(m->d_colidx);
    take(m->d_s); take(m->d_w); take(m->d_zL); take(m->d_zU);
    take(m->d_PQ); take(m->d_cE); take(m->d_cI);
    take(m->d_sigma); take(m->d_D); take(m->d_vals); take(m->d_jtl);
    take(m->d_rhs); take(m->d_dir); take(m->d_dzL); take(m->d_dzU);
    take(m->d_ds); take(m->d_dw); take(m->d_red);
    cudaStream_t ust = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&ust, cudaStreamNonBlocking);
    auto up = [&](void* d, const void* h, size_t b) {
        if (e == cudaSuccess && b) e = cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, ust);
    };
    up(m->d_Pd, h_Pd, 8 * (size_t)B);
    up(m->d_Qd, h_Qd, 8 * (size_t)B);
    up(m->d_lo, lo.data(), 8 * nd);
    up(m->d_hi, hi.data(), 8 * nd);
    up(m->d_u, u.data(), 8 * ndu);
    up(m->d_bus_ptr, bus_ptr.data(), 4 * (size_t)(B + 1));
    up(m->d_bus_end, bus_end.data(), 4 * (size_t)(2 * L));
    up(m->d_gen_of_bus, gen_of_bus.data(), 4 * (size_t)B);
    up(m->d_rowptr, m->rowptr.data(), 4 * (size_t)(n + 1));
    up(m->d_colidx, m->colidx.data(), 4 * (size_t)m->nnz);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ust);
    if (ust) cudaStreamDestroy(ust);
    return e == cudaSuccess ? KKT_OK : KKT_E_CUDA;
}

kkt_status kkt_ipm_solve(kkt_model* m, kkt_ctx* ctx, const kkt_ipm_options* opt_in, double* d_x, double* d_lam,
                         kkt_ipm_info* info, void* stream)
{
    if (!m || !ctx || !d_x || !d_lam) return KKT_E_ARG;
    if (!m->ipm_base) return KKT_E_STATE;
    kkt_ipm_options o;
    if (opt_in) o = *opt_in; else kkt_ipm_default_options(&o);
    if (!(o.tol > 0.0) || o.max_iter < 0 || !(o.mu0 > 0.0) || !(o.kappa_mu > 0.0 && o.kappa_mu < 1.0) ||
        !(o.theta_mu > 1.0) || !(o.tau_min > 0.0 && o.tau_min < 1.0) || !(o.push > 0.0 && o.push < 0.5) ||
        !(o.lin_tol > 0.0) || !(o.delta_w >= 0.0) || !(o.delta_c >= 0.0) || o.angle_ref < 0 ||
        o.angle_ref >= m->nb || !(o.angle_pin >= 0.0))
        return KKT_E_ARG;
    kkt_plan_info pi;
    if (kkt_get_plan(ctx, &pi) != KKT_OK || pi.n != m->n || pi.nnz != m->nnz || pi.batch != 1) return KKT_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int B = m->nb, L = m->nl, G = m->ng, np = m->n_primal, n = m->n, md = n - np, mE = 2 * B;
    const int mI = m->flow ? 2 * L : 0;
    const int blocks = kIpmBlocks, T = kIpmThreads;
    const int iref = B + o.angle_ref;
    const double pin2 = 2.0 * o.angle_pin;
    double* x = d_x;
    double* lam = d_lam;
    double* lamI = lam + mE;
    double* pin = m->ipm_pin;
    double* out = m->d_red + (size_t)kIpmBlocks * kIpmRed;
    auto evaluate = [&]() {
        if (L) ipm_flows_kernel<<<blocks, T, 0, st>>>(L, m->d_f, m->d_t, m->d_g, m->d_b, x, x + B, m->d_PQ);
        ipm_constraints_kernel<<<blocks, T, 0, st>>>(B, L, m->flow, m->d_bus_ptr, m->d_bus_end, m->d_gen_of_bus,
                                                     x + 2 * B, x + 2 * B + G, m->d_Pd, m->d_Qd, m->d_PQ, m->d_cE,
                                                     m->d_cI);
    };
    auto reduce = [&](int min_mask, int sum_mask) -> cudaError_t {
        ipm_final_kernel<<<1, 32, 0, st>>>(blocks, m->d_red, min_mask, sum_mask, out);
        cudaError_t e = cudaMemcpyAsync(pin, out, kIpmRed * sizeof(double), cudaMemcpyDeviceToHost, st);
        return e ? e : cudaStreamSynchronize(st);
    };
    // start
    ipm_push_kernel<<<blocks, T, 0, st>>>(np, o.push, m->d_lo, m->d_hi, x);
    evaluate();
    ipm_start_kernel<<<blocks, T, 0, st>>>(np, md, mI, o.mu0, o.push, x, m->d_lo, m->d_hi, m->d_cI, m->d_u, lam,
                                           m->d_s, m->d_w, m->d_zL, m->d_zU);
    if (cudaGetLastError() != cudaSuccess) return KKT_E_CUDA;
    double mu = o.mu0;
    kkt_ipm_info res{};
    res.status = KKT_E_NOCONV;
    int it = 0;
    for (it = 0;; ++it) {
        evaluate();
        ipm_diag_kernel<<<blocks, T, 0, st>>>(np, md, mE, iref, pin2, x, m->d_lo, m->d_hi, m->d_zL, m->d_zU, m->d_s, m->d_w,
                                              m->d_sigma, m->d_D);
        kkt_status s = kkt_model_assemble(m, x, x + B, lam, m->d_sigma, m->d_D, o.delta_w, o.delta_c, m->d_vals, st);
        if (s != KKT_OK) return s;
        ipm_jtlam_kernel<<<blocks, T, 0, st>>>(np, m->d_rowptr, m->d_colidx, m->d_vals, lam, m->d_jtl);
        ipm_errors_kernel<<<blocks, T, 0, st>>>(np, B, G, mI, iref, pin2, x, m->d_lo, m->d_hi, m->d_zL, m->d_zU, m->d_twoc2,
                                                m->d_jtl, m->d_cE, m->d_cI, m->d_s, m->d_w, m->d_u, lamI, m->d_red);
        if (reduce(1 << 5, 1 << 6) != cudaSuccess) return KKT_E_CUDA;
        const double dual = pin[0], pE = pin[1], pI = pin[2], ds = pin[3], cmax = pin[4], cmin = pin[5];
        res.objective = pin[6];
        const double base = std::max(std::max(dual, pE), std::max(pI, ds));
        auto err = [&](double mu_) { return std::max(base, std::max(cmax - mu_, mu_ - std::min(cmin, cmax))); };
        const double e0 = std::max(base, cmax);
        res.err = e0;
        if (!std::isfinite(e0)) { res.status = KKT_E_NUMERIC; break; }
        if (e0 <= o.tol) { res.status = KKT_OK; break; }
        if (it >= o.max_iter) break;
        while (err(mu) <= o.kappa_eps * mu && mu > o.tol / 10)
            mu = std::max(o.tol / 10, std::min(o.kappa_mu * mu, std::pow(mu, o.theta_mu)));
        ipm_rhs_kernel<<<blocks, T, 0, st>>>(np, B, G, mI, iref, pin2, mu, x, m->d_lo, m->d_hi, m->d_twoc2, m->d_jtl, m->d_cE,
                                             m->d_cI, m->d_s, m->d_w, m->d_u, lamI, m->d_rhs);
        kkt_info li{};
        s = kkt_refactor_refine(ctx, m->d_vals, m->d_rhs, m->d_dir, o.lin_tol, &li, st);
        if (s == KKT_E_NOCONV) res.lin_noconv++;
        else if (s != KKT_OK) { res.status = s; break; }
        res.lin_iters += li.iters;
        res.lin_omega_max = std::max(res.lin_omega_max, li.backward_err);
        const double tau = std::max(o.tau_min, 1.0 - mu);
        ipm_step_kernel<<<blocks, T, 0, st>>>(np, mI, mE, mu, tau, x, m->d_lo, m->d_hi, m->d_zL, m->d_zU, m->d_s,
                                              m->d_w, lamI, m->d_dir, m->d_dzL, m->d_dzU, m->d_ds, m->d_dw,
                                              m->d_red);
        if (reduce(3, 0) != cudaSuccess) return KKT_E_CUDA;
        const double ap = std::min(1.0, pin[0]), ad = std::min(1.0, pin[1]);
        if (!(ap > 0.0) || !(ad > 0.0)) { res.status = KKT_E_NUMERIC; break; }
        ipm_update_kernel<<<blocks, T, 0, st>>>(np, md, mI, ap, ad, x, lam, m->d_s, m->d_w, m->d_zL, m->d_zU,
                                                m->d_dir, m->d_dzL, m->d_dzU, m->d_ds, m->d_dw);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return KKT_E_CUDA;
    res.iters = it;
    res.mu = mu;
    if (info) *info = res;
    return (kkt_status)res.status;
}

}  // extern "C"
