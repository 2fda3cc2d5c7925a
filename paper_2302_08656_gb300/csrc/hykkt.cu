// Saddle-point specialised solve of a KKT system (Sec. V names such a solver
// as a way forward without giving its method; this is the hybrid
// direct-iterative approach to ACOPF KKT systems, see kkt.h):
//
//   K = [ H    J_E^T  J_I^T ]   unknowns (x, y_E, y_I): primal, equality duals,
//       [ J_E -D_E    0     ]   inequality duals; D_E, D_I diagonal
//       [ J_I  0     -D_I   ]
//
// condense the inequality rows (H' = H + J_I^T D_I^{-1} J_I), augment with
// gamma J_E^T J_E (H_g = H' + gamma J_E^T J_E, factored by the library's own
// multifrontal LU in an inner context), solve the equality duals by conjugate
// gradients on the symmetric operator C^{1/2} J_E H_g^{-1} J_E^T C^{1/2} + D_E
// (C = I - gamma D_E; one solve with H_g per iteration, x updated along),
// then recover y_E and y_I. Every step runs in kernels on the caller's stream; the host reads the
// conjugate-gradient residual after every iteration to stop.
#include "../../include/kkt.h"
#include "hykkt_plan.hpp"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 304;          // 2 x 152 SMs, grid-stride loops; also the partial sums of a dot product

using kktgb::HgTerm;

__global__ void hg_assemble_kernel(int64_t nnz_g, const int64_t* __restrict__ cptr, const HgTerm* __restrict__ cl,
                                   const double* __restrict__ vals, const double* __restrict__ dinv, double gamma,
                                   double* __restrict__ hg)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz_g; e += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int64_t c = cptr[e]; c < cptr[e + 1]; ++c) {
            const HgTerm t = cl[c];
            if (t.k == -1) acc += vals[t.a];
            else if (t.k == -2) acc += gamma * (vals[t.a] * vals[t.b]);
            else acc += (vals[t.a] * vals[t.b]) * dinv[t.k];
        }
        hg[e] = acc;
    }
}

// the (2,2) block: d_E, C = 1 - gamma d_E and its square root, 1 / d_I; flag
// (bit 0: some d_I <= 0 or not finite, bit 1: some C <= 0)
__global__ void duals_kernel(int mE, int mI, const int* __restrict__ dpos, const double* __restrict__ vals,
                             double gamma, double* __restrict__ dE, double* __restrict__ C, double* __restrict__ sq,
                             double* __restrict__ dinv, int* __restrict__ flag)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < mE + mI; k += gridDim.x * blockDim.x) {
        const double d = -vals[dpos[k]];
        if (k < mE) {
            const double c = 1.0 - gamma * d;
            dE[k] = d;
            C[k] = c;
            sq[k] = sqrt(c);
            if (!(c > 0.0)) atomicOr(flag, 2);
        } else {
            dinv[k - mE] = 1.0 / d;
            if (!(d > 0.0) || !isfinite(d)) atomicOr(flag, 1);
        }
    }
}

// y = J x over the rows of a block (CSR of positions into K's values)
__global__ void j_mul_kernel(int m, const int* __restrict__ ptr, const int* __restrict__ col,
                             const int* __restrict__ pos, const double* __restrict__ vals, const double* __restrict__ x,
                             double* __restrict__ y)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int p = ptr[r]; p < ptr[r + 1]; ++p) acc += vals[pos[p]] * x[col[p]];
        y[r] = acc;
    }
}

// out = base + J_I^T (xi .* si) + ge J_E^T (xe .* se) over the primal rows
// (transposes as CSR of positions); base, xi, xe, si, se may be null (a null
// scale is 1)
__global__ void jt_mul_kernel(int np, const int* __restrict__ ip, const int* __restrict__ ic, const int* __restrict__ ipos,
                              const int* __restrict__ ep, const int* __restrict__ ec, const int* __restrict__ epos,
                              const double* __restrict__ vals, const double* __restrict__ base,
                              const double* __restrict__ xi, const double* __restrict__ si,
                              const double* __restrict__ xe, const double* __restrict__ se, double ge,
                              double* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        double a = 0.0, e = 0.0;
        if (xi)
            for (int p = ip[i]; p < ip[i + 1]; ++p) {
                const int k = ic[p];
                a += vals[ipos[p]] * (si ? xi[k] * si[k] : xi[k]);
            }
        if (xe)
            for (int p = ep[i]; p < ep[i + 1]; ++p) {
                const int k = ec[p];
                e += vals[epos[p]] * (se ? xe[k] * se[k] : xe[k]);
            }
        out[i] = (base ? base[i] : 0.0) + a + ge * e;
    }
}

// small vector steps of the method, by `op`
__global__ void vec_kernel(int op, int n, const double* __restrict__ a, const double* __restrict__ b,
                           const double* __restrict__ c, double* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        switch (op) {
        case 1: out[i] = a[i] * (b[i] - c[i]); break;             // b' = sq .* (J_E t - r_E)
        case 3: out[i] = a[i] / b[i]; break;                      // y_E = w ./ sq
        default: out[i] = (a[i] - b[i]) * c[i]; break;            // y_I = (J_I x - r_I) .* (1 / d_I)
        }
    }
}

// partial dot products (fixed order: block b sums i = b*T + t, + grid stride)
__global__ void dot_part_kernel(int n, const double* __restrict__ a, const double* __restrict__ b,
                                double* __restrict__ part)
{
    __shared__ double s[kThreads];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc += a[i] * b[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void dot_final_kernel(const double* __restrict__ part, double* __restrict__ out)
{
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int b = 0; b < kBlocks; ++b) acc += part[b];
        *out = acc;
    }
}

// sum of the kBlocks partials, the same fixed order in every block (warp 0:
// strided lane sums, then a shuffle tree); every thread gets the result
__device__ double sum_parts(const double* __restrict__ part)
{
    __shared__ double res;
    if (threadIdx.x < 32) {
        double a = 0.0;
        for (int b = threadIdx.x; b < kBlocks; b += 32) a += part[b];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (threadIdx.x == 0) res = a;
    }
    __syncthreads();
    const double v = res;
    __syncthreads();
    return v;
}

__device__ void block_sum_to(double acc, double* __restrict__ part)
{
    __shared__ double s[kThreads];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// one conjugate-gradient iteration in three kernels (kBlocks blocks each; the
// scalars stay on the device; s[cur] = r.r of this iteration, the next one
// goes to s[cur ^ 1]):
//   q = sq .* (J_E v) + d_E .* p, partial p.q     (v = H_g^{-1} J_E^T (sq .* p))
__global__ void __launch_bounds__(kThreads) cg_q_kernel(int m, const int* __restrict__ ptr, const int* __restrict__ col,
                                                        const int* __restrict__ pos, const double* __restrict__ vals,
                                                        const double* __restrict__ v, const double* __restrict__ sq,
                                                        const double* __restrict__ dE, const double* __restrict__ p,
                                                        double* __restrict__ q, double* __restrict__ part)
{
    double acc = 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
        double jv = 0.0;
        for (int k = ptr[r]; k < ptr[r + 1]; ++k) jv += vals[pos[k]] * v[col[k]];
        const double qr = sq[r] * jv + dE[r] * p[r];
        q[r] = qr;
        acc += p[r] * qr;
    }
    block_sum_to(acc, part);
}

//   alpha = s[cur] / (p.q); w += alpha p; r -= alpha q; x -= alpha v
//   (x = H_g^{-1} (r'' - J_E^T (sq .* w)) kept along); partial r.r
__global__ void __launch_bounds__(kThreads) cg_update_kernel(int m, int np, const double* __restrict__ part_pq,
                                                             const double* __restrict__ s, int cur,
                                                             const double* __restrict__ p, const double* __restrict__ q,
                                                             const double* __restrict__ v, double* __restrict__ w,
                                                             double* __restrict__ r, double* __restrict__ x,
                                                             double* __restrict__ part_rr)
{
    const double alpha = s[cur] / sum_parts(part_pq);
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        w[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        acc += ri * ri;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) x[i] -= alpha * v[i];
    block_sum_to(acc, part_rr);
}

//   s[cur ^ 1] = r.r; p = r + (s[cur ^ 1] / s[cur]) p
__global__ void __launch_bounds__(kThreads) cg_direction_kernel(int m, const double* __restrict__ part_rr, double* s,
                                                                int cur, const double* __restrict__ r,
                                                                double* __restrict__ p)
{
    const double rr = sum_parts(part_rr);
    const double beta = rr / s[cur];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) p[i] = r[i] + beta * p[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) s[cur ^ 1] = rr;
}

__device__ __forceinline__ unsigned long long mag(double v)
{
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// per block: max |b - K z|, |z|, |b|, sum_j |K_ij| over the rows (bit patterns:
// NaN sorts above +Inf)
__global__ void resid_part_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                  const double* __restrict__ vals, const double* __restrict__ z,
                                  const double* __restrict__ b, unsigned long long* __restrict__ part)
{
    __shared__ unsigned long long s[4][kThreads];
    unsigned long long m[4] = {0ull, 0ull, 0ull, 0ull};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = 0.0, rs = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            acc += vals[p] * z[ci[p]];
            rs += fabs(vals[p]);
        }
        const unsigned long long v[4] = {mag(b[i] - acc), mag(z[i]), mag(b[i]), mag(rs)};
        for (int q = 0; q < 4; ++q) m[q] = v[q] > m[q] ? v[q] : m[q];
    }
    for (int q = 0; q < 4; ++q) s[q][threadIdx.x] = m[q];
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 4; ++q) s[q][threadIdx.x] = s[q][threadIdx.x + o] > s[q][threadIdx.x] ? s[q][threadIdx.x + o] : s[q][threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x < 4) part[blockIdx.x * 4 + threadIdx.x] = s[threadIdx.x][0];
}

template <typename X>
X* dev_alloc(size_t count, cudaError_t& e)
{
    void* p = nullptr;
    if (e == cudaSuccess && count) e = cudaMalloc(&p, count * sizeof(X));
    return static_cast<X*>(p);
}

template <typename X>
cudaError_t upload(X* dst, const std::vector<X>& src)
{
    return src.empty() ? cudaSuccess : cudaMemcpy(dst, src.data(), src.size() * sizeof(X), cudaMemcpyHostToDevice);
}

}  // namespace

struct kkt_hykkt {
    int n = 0, np = 0, mE = 0, mI = 0;
    int64_t nnz = 0, nnz_g = 0;
    double gamma = 0.0;
    kkt_ctx* inner = nullptr;
    // K and the blocks (positions into K's values)
    int *rp = nullptr, *ci = nullptr, *dpos = nullptr;
    int *je_p = nullptr, *je_c = nullptr, *je_v = nullptr, *ji_p = nullptr, *ji_c = nullptr, *ji_v = nullptr;
    int *jet_p = nullptr, *jet_c = nullptr, *jet_v = nullptr, *jit_p = nullptr, *jit_c = nullptr, *jit_v = nullptr;
    int64_t* cptr = nullptr;
    HgTerm* cl = nullptr;
    double* hg = nullptr;
    // vectors and scalars
    double *dE = nullptr, *C = nullptr, *sq = nullptr, *dinv = nullptr;
    double *r2 = nullptr, *u = nullptr, *v = nullptr;                      // np
    double *w = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *e = nullptr;   // mE
    double *part = nullptr, *part2 = nullptr, *s = nullptr;
    unsigned long long* rpart = nullptr;
    int* flag = nullptr;
    double* pin = nullptr;                                       // host: s[0..3], flag, residual partials
};

extern "C" {

kkt_status kkt_hykkt_analyze(int32_t n, int32_t n_primal, int32_t m_eq, const int32_t* h_rowptr,
                             const int32_t* h_colidx, double gamma, kkt_hykkt** out)
{
    if (!out || !h_rowptr || !h_colidx || n <= 0 || n_primal <= 0 || m_eq <= 0 || n_primal + m_eq > n ||
        !(gamma >= 0.0) || !std::isfinite(gamma))
        return KKT_E_ARG;
    *out = nullptr;
    const int np = n_primal, mE = m_eq, mI = n - n_primal - m_eq;
    const int64_t nnz = h_rowptr[n];
    kktgb::HykktPlan pl;
    if (kktgb::build_hykkt_plan(n, np, mE, h_rowptr, h_colidx, pl) != 0) return KKT_E_STRUCT;
    const std::vector<int>&dpos = pl.dpos, &je_p = pl.je_p, &je_c = pl.je_c, &je_v = pl.je_v, &ji_p = pl.ji_p,
                          &ji_c = pl.ji_c, &ji_v = pl.ji_v, &jet_p = pl.jet_p, &jet_c = pl.jet_c, &jet_v = pl.jet_v,
                          &jit_p = pl.jit_p, &jit_c = pl.jit_c, &jit_v = pl.jit_v, &hg_p = pl.hg_p, &hg_c = pl.hg_c;
    const std::vector<int64_t>& cptr = pl.term_ptr;
    const std::vector<HgTerm>& cl = pl.term;
    kkt_hykkt* h = new (std::nothrow) kkt_hykkt();
    if (!h) return KKT_E_NOMEM;
    h->n = n; h->np = np; h->mE = mE; h->mI = mI; h->nnz = nnz; h->nnz_g = (int64_t)hg_c.size(); h->gamma = gamma;
    kkt_options opt;
    kkt_default_options(&opt);
    opt.precision = KKT_FP64;
    kkt_status st = kkt_analyze(np, np, hg_p.data(), hg_c.data(), nullptr, &opt, &h->inner);
    if (st != KKT_OK) {
        delete h;
        return st;
    }
    cudaError_t e = cudaSuccess;
    h->rp = dev_alloc<int>(n + 1, e); h->ci = dev_alloc<int>(nnz, e); h->dpos = dev_alloc<int>(mE + mI, e);
    h->je_p = dev_alloc<int>(je_p.size(), e); h->je_c = dev_alloc<int>(je_c.size(), e); h->je_v = dev_alloc<int>(je_v.size(), e);
    h->ji_p = dev_alloc<int>(ji_p.size(), e); h->ji_c = dev_alloc<int>(ji_c.size(), e); h->ji_v = dev_alloc<int>(ji_v.size(), e);
    h->jet_p = dev_alloc<int>(jet_p.size(), e); h->jet_c = dev_alloc<int>(jet_c.size(), e); h->jet_v = dev_alloc<int>(jet_v.size(), e);
    h->jit_p = dev_alloc<int>(jit_p.size(), e); h->jit_c = dev_alloc<int>(jit_c.size(), e); h->jit_v = dev_alloc<int>(jit_v.size(), e);
    h->cptr = dev_alloc<int64_t>(cptr.size(), e); h->cl = dev_alloc<HgTerm>(cl.size(), e);
    h->hg = dev_alloc<double>(hg_c.size(), e);
    h->dE = dev_alloc<double>(mE, e); h->C = dev_alloc<double>(mE, e); h->sq = dev_alloc<double>(mE, e);
    h->dinv = dev_alloc<double>(std::max(mI, 1), e);
    h->r2 = dev_alloc<double>(np, e); h->u = dev_alloc<double>(np, e);
    h->v = dev_alloc<double>(np, e);
    h->w = dev_alloc<double>(mE, e); h->r = dev_alloc<double>(mE, e); h->p = dev_alloc<double>(mE, e);
    h->q = dev_alloc<double>(mE, e); h->e = dev_alloc<double>(std::max(mE, mI), e);
    h->part = dev_alloc<double>(kBlocks, e); h->part2 = dev_alloc<double>(kBlocks, e);
    h->s = dev_alloc<double>(4, e);
    h->rpart = dev_alloc<unsigned long long>(4 * kBlocks, e);
    h->flag = dev_alloc<int>(1, e);
    if (e == cudaSuccess) e = cudaMallocHost(&h->pin, sizeof(double) * (8 + 4 * kBlocks));
    if (e == cudaSuccess) e = cudaMemcpy(h->rp, h_rowptr, (n + 1) * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->ci, h_colidx, nnz * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = upload(h->dpos, dpos);
    if (e == cudaSuccess) e = upload(h->je_p, je_p);
    if (e == cudaSuccess) e = upload(h->je_c, je_c);
    if (e == cudaSuccess) e = upload(h->je_v, je_v);
    if (e == cudaSuccess) e = upload(h->ji_p, ji_p);
    if (e == cudaSuccess) e = upload(h->ji_c, ji_c);
    if (e == cudaSuccess) e = upload(h->ji_v, ji_v);
    if (e == cudaSuccess) e = upload(h->jet_p, jet_p);
    if (e == cudaSuccess) e = upload(h->jet_c, jet_c);
    if (e == cudaSuccess) e = upload(h->jet_v, jet_v);
    if (e == cudaSuccess) e = upload(h->jit_p, jit_p);
    if (e == cudaSuccess) e = upload(h->jit_c, jit_c);
    if (e == cudaSuccess) e = upload(h->jit_v, jit_v);
    if (e == cudaSuccess) e = upload(h->cptr, cptr);
    if (e == cudaSuccess) e = upload(h->cl, cl);
    if (e != cudaSuccess) {
        kkt_hykkt_destroy(h);
        return e == cudaErrorMemoryAllocation ? KKT_E_NOMEM : KKT_E_CUDA;
    }
    *out = h;
    return KKT_OK;
}

}  // extern "C"

namespace {

void dot(const kkt_hykkt* h, int n, const double* a, const double* b, double* out, cudaStream_t st)
{
    dot_part_kernel<<<kBlocks, kThreads, 0, st>>>(n, a, b, h->part);
    dot_final_kernel<<<1, 32, 0, st>>>(h->part, out);
}

int grid_for(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>(kBlocks * 4, (n + kThreads - 1) / kThreads));
}

}  // namespace

extern "C" {

kkt_status kkt_hykkt_solve(kkt_hykkt* h, const double* d_vals, const double* d_rhs, double* d_z, double tol,
                           int32_t max_iter, kkt_hykkt_info* info, void* stream)
{
    if (!h || !d_vals || !d_rhs || !d_z || d_rhs == d_z || !(tol >= 0.0) || max_iter < 0) return KKT_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int np = h->np, mE = h->mE, mI = h->mI;
    const double* rx = d_rhs;
    const double* rE = d_rhs + np;
    const double* rI = d_rhs + np + mE;
    double* x = d_z;
    double* yE = d_z + np;
    double* yI = d_z + np + mE;
    const int gE = grid_for(mE), gI = grid_for(mI), gP = grid_for(np);
#define HK_CUDA(call)                                                                                             \
    do {                                                                                                          \
        if ((call) != cudaSuccess) return KKT_E_CUDA;                                                             \
    } while (0)
    kkt_status ks;
    int nl = 0;                                                   // kernels launched here
    kkt_info inner0;
    kkt_get_info(h->inner, &inner0);
    // the (2,2) block, H_g and its factorization
    HK_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), st));
    duals_kernel<<<grid_for(mE + mI), kThreads, 0, st>>>(mE, mI, h->dpos, d_vals, h->gamma, h->dE, h->C, h->sq,
                                                          h->dinv, h->flag);
    ++nl;
    hg_assemble_kernel<<<grid_for(h->nnz_g), kThreads, 0, st>>>(h->nnz_g, h->cptr, h->cl, d_vals, h->dinv, h->gamma,
                                                                 h->hg);
    ++nl;
    HK_CUDA(cudaGetLastError());
    if ((ks = kkt_refactor(h->inner, h->hg, st)) != KKT_OK) return ks;
    // r'' = r_x + J_I^T (r_I ./ d_I) + gamma J_E^T r_E; x starts at t = H_g^{-1} r''
    jt_mul_kernel<<<gP, kThreads, 0, st>>>(np, h->jit_p, h->jit_c, h->jit_v, h->jet_p, h->jet_c, h->jet_v, d_vals, rx,
                                           mI ? rI : nullptr, h->dinv, rE, nullptr, h->gamma, h->r2);
    ++nl;
    HK_CUDA(cudaGetLastError());
    if ((ks = kkt_solve(h->inner, h->r2, x, st)) != KKT_OK) return ks;
    // right-hand side of the reduced system: b' = sq .* (J_E t - r_E); w = 0, r = p = b'
    j_mul_kernel<<<gE, kThreads, 0, st>>>(mE, h->je_p, h->je_c, h->je_v, d_vals, x, h->q);
    ++nl;
    vec_kernel<<<gE, kThreads, 0, st>>>(1, mE, h->sq, h->q, rE, h->r);
    ++nl;
    HK_CUDA(cudaMemsetAsync(h->w, 0, sizeof(double) * mE, st));
    HK_CUDA(cudaMemcpyAsync(h->p, h->r, sizeof(double) * mE, cudaMemcpyDeviceToDevice, st));
    dot(h, mE, h->r, h->r, h->s, st);
    nl += 2;
    HK_CUDA(cudaGetLastError());
    // conjugate gradients on (C^{1/2} J_E H_g^{-1} J_E^T C^{1/2} + D_E) w = b';
    // each iteration costs a whole solve with H_g, so the host reads r.r after
    // every one (a short copy and wait) instead of running past convergence
    int it = 0, cur = 0;
    double nb2 = -1.0, rr = 0.0;
    for (;; ++it) {
        HK_CUDA(cudaMemcpyAsync(h->pin, h->s + cur, sizeof(double), cudaMemcpyDeviceToHost, st));
        if (it == 0) HK_CUDA(cudaMemcpyAsync(h->pin + 1, h->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        HK_CUDA(cudaStreamSynchronize(st));
        if (it == 0) {
            int fl = 0;
            std::memcpy(&fl, h->pin + 1, sizeof(int));
            if (fl) return KKT_E_NUMERIC;                       // d_I <= 0 or gamma d_E >= 1
        }
        rr = h->pin[0];
        if (nb2 < 0.0) nb2 = rr;
        if (!(rr == rr) || !std::isfinite(rr)) return KKT_E_NUMERIC;
        if (std::sqrt(rr) <= tol * std::sqrt(nb2) || it >= max_iter) break;
        // v = H_g^{-1} J_E^T (sq .* p)
        jt_mul_kernel<<<gP, kThreads, 0, st>>>(np, h->jit_p, h->jit_c, h->jit_v, h->jet_p, h->jet_c, h->jet_v, d_vals,
                                               nullptr, nullptr, nullptr, h->p, h->sq, 1.0, h->u);
        ++nl;
        HK_CUDA(cudaGetLastError());
        if ((ks = kkt_solve(h->inner, h->u, h->v, st)) != KKT_OK) return ks;
        cg_q_kernel<<<kBlocks, kThreads, 0, st>>>(mE, h->je_p, h->je_c, h->je_v, d_vals, h->v, h->sq, h->dE, h->p,
                                                  h->q, h->part);
        cg_update_kernel<<<kBlocks, kThreads, 0, st>>>(mE, np, h->part, h->s, cur, h->p, h->q, h->v, h->w, h->r, x,
                                                       h->part2);
        cg_direction_kernel<<<kBlocks, kThreads, 0, st>>>(mE, h->part2, h->s, cur, h->r, h->p);
        nl += 3;
        HK_CUDA(cudaGetLastError());
        cur ^= 1;
    }
    // recover: y_E = w ./ sq (x kept along the iteration), y_I = (J_I x - r_I) ./ d_I
    vec_kernel<<<gE, kThreads, 0, st>>>(3, mE, h->w, h->sq, nullptr, yE);
    ++nl;
    if (mI) {
        j_mul_kernel<<<gI, kThreads, 0, st>>>(mI, h->ji_p, h->ji_c, h->ji_v, d_vals, x, h->e);
        ++nl;
        vec_kernel<<<gI, kThreads, 0, st>>>(5, mI, h->e, rI, h->dinv, yI);
        ++nl;
    }
    // backward error of z for K
    resid_part_kernel<<<kBlocks, kThreads, 0, st>>>(h->n, h->rp, h->ci, d_vals, d_z, d_rhs, h->rpart);
    ++nl;
    HK_CUDA(cudaGetLastError());
    HK_CUDA(cudaMemcpyAsync(h->pin + 8, h->rpart, sizeof(unsigned long long) * 4 * kBlocks, cudaMemcpyDeviceToHost, st));
    HK_CUDA(cudaStreamSynchronize(st));
    unsigned long long m[4] = {0ull, 0ull, 0ull, 0ull};
    const unsigned long long* hp = reinterpret_cast<const unsigned long long*>(h->pin + 8);
    for (int b = 0; b < kBlocks; ++b)
        for (int k = 0; k < 4; ++k) m[k] = std::max(m[k], hp[4 * b + k]);
    double v[4];
    std::memcpy(v, m, sizeof(v));
    const double den = v[3] * v[1] + v[2];
    const double omega = den > 0.0 ? v[0] / den : (den == 0.0 ? v[0] : den);
    kkt_info inner_info;
    kkt_get_info(h->inner, &inner_info);
    const bool converged = std::sqrt(rr) <= tol * std::sqrt(nb2 > 0.0 ? nb2 : 0.0) || nb2 == 0.0;
    if (info) {
        info->cg_iters = it;
        info->status = converged ? KKT_OK : KKT_E_NOCONV;
        info->cg_resid = nb2 > 0.0 ? std::sqrt(rr / nb2) : 0.0;
        info->backward_err = omega;
        info->n_perturbed = inner_info.n_perturbed;
        info->launches = nl + (int)(inner_info.launches - inner0.launches);
    }
#undef HK_CUDA
    return converged ? KKT_OK : KKT_E_NOCONV;
}

kkt_status kkt_hykkt_inner(kkt_hykkt* h, kkt_ctx** out)
{
    if (!h || !out) return KKT_E_ARG;
    *out = h->inner;
    return KKT_OK;
}

void kkt_hykkt_destroy(kkt_hykkt* h)
{
    if (!h) return;
    if (h->inner) kkt_destroy(h->inner);
    void* dev[] = {h->rp, h->ci, h->dpos, h->je_p, h->je_c, h->je_v, h->ji_p, h->ji_c, h->ji_v, h->jet_p, h->jet_c,
                   h->jet_v, h->jit_p, h->jit_c, h->jit_v, h->cptr, h->cl, h->hg, h->dE, h->C, h->sq, h->dinv, h->r2,
                   h->u, h->v, h->w, h->r, h->p, h->q, h->e, h->part, h->part2, h->s, h->rpart, h->flag};
    for (void* p : dev)
        if (p) cudaFree(p);
    if (h->pin) cudaFreeHost(h->pin);
    delete h;
}

}  // extern "C"
