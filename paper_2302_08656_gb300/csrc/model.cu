// GPU assembly of the ACOPF KKT values K_k (Eq. 11) from the interior-point
// iterate: the model evaluation step that precedes the linear solve in every
// Newton iteration. The paper measures it at about 30 % of the CPU run time
// (Sec. III) and projects a 2x overall gain from moving it to the GPU
// (Sec. IV); here it writes the CSR values that kkt_refactor consumes, so an
// iteration's inputs to the GPU shrink from nnz(K) values to the iterate.
//
// Model (Eqs. 1-4 in polar voltages, no shunts, unit taps):
//   primal x = (|V|_1..|V|_B, theta_1..theta_B, Pg_1..Pg_G, Qg_1..Qg_G);
//   equalities: active / reactive power balance per bus, with the flow
//     leaving bus i on line (i, j) of admittance y = g + jb = 1 / (r + jx)
//       P_ij = g V_i^2 - V_i V_j (g cos t + b sin t)
//       Q_ij = -b V_i^2 - V_i V_j (g sin t - b cos t),   t = theta_i - theta_j
//     entering the balance of bus i with a minus sign, generators with +1;
//   inequalities (optional): P_ij^2 + Q_ij^2 <= S^2 at both line ends;
//   objective: sum c2 Pg^2.
// K = [[H + Sigma + dw I, J^T], [J, -dc I]] with H the Hessian of the
// Lagrangian F + lambda^T c (balance rows, then the flow rows of the two
// ends), Sigma the barrier diagonal (zero on angles, supplied by the caller).
//
// Two kernels: one thread per line evaluates the line's 40 terms (its 4 x 4
// Hessian block, the 16 balance-Jacobian entries of its two ends, the 8
// flow-limit Jacobian entries); one thread per nonzero of K then sums the
// terms that land on it, in a fixed order, and adds its diagonal or constant
// part. No atomics: the result is deterministic.
#include "../../include/kkt.h"
#include "model.hpp"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

namespace {

constexpr int kLineTerms = 40;     // 16 Hessian + 16 balance Jacobian + 8 flow Jacobian

// kind of the diagonal / constant part of a nonzero
enum : int { kExtraNone = 0, kExtraPrimal = 1, kExtraDual = 2, kExtraOne = 3 };

__global__ void __launch_bounds__(128) line_terms_kernel(int nb, int nl, int flow, const int* __restrict__ lf,
                                                         const int* __restrict__ lt, const double* __restrict__ lg,
                                                         const double* __restrict__ lb, const double* __restrict__ V,
                                                         const double* __restrict__ th,
                                                         const double* __restrict__ lam, double* __restrict__ out)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    const int i = lf[l], j = lt[l];
    const double g = lg[l], b = lb[l];
    const double Vi = V[i], Vj = V[j];
    const double t = th[i] - th[j];
    const double c = cos(t), s = sin(t);
    // end e = 0: flow leaving i (variables in order Vi, Vj, ti, tj);
    // end e = 1: flow leaving j, written back in the same variable order
    double P[2], Q[2], dP[2][4], dQ[2][4], HP[2][4][4], HQ[2][4][4];
    for (int e = 0; e < 2; ++e) {
        const double Va = e ? Vj : Vi, Vb = e ? Vi : Vj;
        const double sa = e ? -s : s;                       // sin of (theta_a - theta_b)
        const double A = g * c + b * sa;                    // g cos + b sin
        const double Bq = g * sa - b * c;                   // g sin - b cos
        const double VV = Va * Vb;
        // derivatives in the end's own order (Va, Vb, ta, tb)
        const double p[4] = {2.0 * g * Va - Vb * A, -Va * A, VV * Bq, -VV * Bq};
        const double qd[4] = {-2.0 * b * Va - Vb * Bq, -Va * Bq, -VV * A, VV * A};
        double hp[4][4] = {{2.0 * g, -A, Vb * Bq, -Vb * Bq},
                           {-A, 0.0, Va * Bq, -Va * Bq},
                           {Vb * Bq, Va * Bq, VV * A, -VV * A},
                           {-Vb * Bq, -Va * Bq, -VV * A, VV * A}};
        double hq[4][4] = {{-2.0 * b, -Bq, -Vb * A, Vb * A},
                           {-Bq, 0.0, -Va * A, Va * A},
                           {-Vb * A, -Va * A, VV * Bq, -VV * Bq},
                           {Vb * A, Va * A, -VV * Bq, VV * Bq}};
        P[e] = g * Va * Va - VV * A;
        Q[e] = -b * Va * Va - VV * Bq;
        // map (Va, Vb, ta, tb) -> (Vi, Vj, ti, tj): identity for e = 0, swap pairs for e = 1
        for (int x = 0; x < 4; ++x) {
            const int xs = e ? (x ^ 1) : x;
            dP[e][xs] = p[x];
            dQ[e][xs] = qd[x];
            for (int y = 0; y < 4; ++y) {
                const int ys = e ? (y ^ 1) : y;
                HP[e][xs][ys] = hp[x][y];
                HQ[e][xs][ys] = hq[x][y];
            }
        }
    }
    const double lPi = lam[i], lPj = lam[j], lQi = lam[nb + i], lQj = lam[nb + j];
    const double lF = flow ? lam[2 * nb + l] : 0.0, lT = flow ? lam[2 * nb + nl + l] : 0.0;
    double* o = out + (int64_t)l * kLineTerms;
    for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y) {
            double h = -(lPi * HP[0][x][y] + lPj * HP[1][x][y] + lQi * HQ[0][x][y] + lQj * HQ[1][x][y]);
            if (flow) {
                h += lF * 2.0 * (dP[0][x] * dP[0][y] + dQ[0][x] * dQ[0][y] + P[0] * HP[0][x][y] + Q[0] * HQ[0][x][y]);
                h += lT * 2.0 * (dP[1][x] * dP[1][y] + dQ[1][x] * dQ[1][y] + P[1] * HP[1][x][y] + Q[1] * HQ[1][x][y]);
            }
            o[4 * x + y] = h;
        }
    for (int x = 0; x < 4; ++x) {
        o[16 + x] = -dP[0][x];          // P balance of bus i
        o[20 + x] = -dP[1][x];          // P balance of bus j
        o[24 + x] = -dQ[0][x];          // Q balance of bus i
        o[28 + x] = -dQ[1][x];          // Q balance of bus j
        o[32 + x] = 2.0 * (P[0] * dP[0][x] + Q[0] * dQ[0][x]);   // |S|^2 at the i end
        o[36 + x] = 2.0 * (P[1] * dP[1][x] + Q[1] * dQ[1][x]);   // |S|^2 at the j end
    }
}

__global__ void __launch_bounds__(256) gather_values_kernel(int64_t nnz, const int* __restrict__ tptr,
                                                            const int* __restrict__ tidx,
                                                            const int* __restrict__ extra_kind,
                                                            const int* __restrict__ extra_arg,
                                                            const double* __restrict__ terms,
                                                            const double* __restrict__ sigma,
                                                            const double* __restrict__ dual_diag,
                                                            const double* __restrict__ twoc2, int pg0, int ng,
                                                            double dw, double dc, double* __restrict__ vals)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    double acc = 0.0;
    for (int k = tptr[e]; k < tptr[e + 1]; ++k) acc += terms[tidx[k]];
    const int kind = extra_kind[e];
    if (kind == kExtraPrimal) {
        const int i = extra_arg[e];
        double d = sigma[i] + dw;
        if (i >= pg0 && i < pg0 + ng) d += twoc2[i - pg0];
        acc += d;
    } else if (kind == kExtraDual) {
        acc -= dual_diag ? dc + dual_diag[extra_arg[e]] : dc;
    } else if (kind == kExtraOne) {
        acc += 1.0;
    }
    vals[e] = acc;
}

}  // namespace


extern "C" {

kkt_status kkt_model_create(int32_t n_bus, int32_t n_branch, int32_t n_gen, const int32_t* h_from,
                            const int32_t* h_to, const double* h_r, const double* h_x, const int32_t* h_gen_bus,
                            const double* h_c2, int flags, kkt_model** out)
{
    const int flow_limits = flags & KKT_MODEL_FLOW_LIMITS;
    if (flags & ~(KKT_MODEL_FLOW_LIMITS | KKT_MODEL_HOST_ONLY)) return KKT_E_ARG;
    if (!out || n_bus <= 0 || n_branch < 0 || n_gen < 0) return KKT_E_ARG;
    if ((n_branch && (!h_from || !h_to || !h_r || !h_x)) || (n_gen && (!h_gen_bus || !h_c2))) return KKT_E_ARG;
    *out = nullptr;
    const int B = n_bus, L = n_branch, G = n_gen;
    for (int l = 0; l < L; ++l) {
        if (h_from[l] < 0 || h_from[l] >= B || h_to[l] < 0 || h_to[l] >= B || h_from[l] == h_to[l]) return KKT_E_ARG;
        const double z2 = h_r[l] * h_r[l] + h_x[l] * h_x[l];
        if (!(z2 > 0.0) || !std::isfinite(z2)) return KKT_E_ARG;
    }
    for (int k = 0; k < G; ++k)
        if (h_gen_bus[k] < 0 || h_gen_bus[k] >= B) return KKT_E_ARG;
    kkt_model* m = nullptr;
    try {
        m = new kkt_model();
        m->nb = B; m->nl = L; m->ng = G; m->flow = flow_limits ? 1 : 0;
        m->n_primal = 2 * B + 2 * G;
        const int n_dual = 2 * B + (m->flow ? 2 * L : 0);
        const int n = m->n = m->n_primal + n_dual;
        // every (row, column, contribution) of K; contribution >= 0: a line term
        // index, < 0: an extra part encoded as -(1 + kind * 2^29 + arg)... kept apart:
        struct Trip { int r, c, term, kind, arg; };
        std::vector<Trip> tr;
        tr.reserve((size_t)L * 56 + (size_t)n + 4 * (size_t)G);
        const int rP = m->n_primal, rQ = m->n_primal + B, rF = m->n_primal + 2 * B, rT = rF + L;
        for (int l = 0; l < L; ++l) {
            const int i = h_from[l], j = h_to[l];
            const int loc[4] = {i, j, B + i, B + j};
            const int base = l * kLineTerms;
            for (int x = 0; x < 4; ++x)
                for (int y = 0; y < 4; ++y) tr.push_back({loc[x], loc[y], base + 4 * x + y, kExtraNone, 0});
            const int jrow[6] = {rP + i, rP + j, rQ + i, rQ + j, rF + l, rT + l};
            const int nrow = m->flow ? 6 : 4;
            for (int r = 0; r < nrow; ++r)
                for (int x = 0; x < 4; ++x) {
                    tr.push_back({jrow[r], loc[x], base + 16 + 4 * r + x, kExtraNone, 0});
                    tr.push_back({loc[x], jrow[r], base + 16 + 4 * r + x, kExtraNone, 0});
                }
        }
        for (int i = 0; i < m->n_primal; ++i) tr.push_back({i, i, -1, kExtraPrimal, i});
        for (int k = 0; k < G; ++k) {
            const int pg = 2 * B + k, qg = 2 * B + G + k, bus = h_gen_bus[k];
            tr.push_back({rP + bus, pg, -1, kExtraOne, 0});
            tr.push_back({pg, rP + bus, -1, kExtraOne, 0});
            tr.push_back({rQ + bus, qg, -1, kExtraOne, 0});
            tr.push_back({qg, rQ + bus, -1, kExtraOne, 0});
        }
        for (int i = m->n_primal; i < n; ++i) tr.push_back({i, i, -1, kExtraDual, i - m->n_primal});
        std::stable_sort(tr.begin(), tr.end(), [](const Trip& a, const Trip& b) {
            return a.r != b.r ? a.r < b.r : a.c < b.c;
        });
        std::vector<int> tptr(1, 0), tidx, kind, arg;
        m->rowptr.assign(n + 1, 0);
        for (size_t p = 0; p < tr.size();) {
            size_t q = p;
            int kd = kExtraNone, ag = 0;
            while (q < tr.size() && tr[q].r == tr[p].r && tr[q].c == tr[p].c) {
                if (tr[q].term >= 0) tidx.push_back(tr[q].term);
                else if (kd == kExtraNone) { kd = tr[q].kind; ag = tr[q].arg; }
                else return delete m, KKT_E_ARG;                     // two generators on one bus pair
                ++q;
            }
            m->colidx.push_back(tr[p].c);
            m->rowptr[tr[p].r + 1]++;
            tptr.push_back((int)tidx.size());
            kind.push_back(kd);
            arg.push_back(ag);
            p = q;
        }
        for (int r = 0; r < n; ++r) m->rowptr[r + 1] += m->rowptr[r];
        m->nnz = (int64_t)m->colidx.size();
        std::vector<double> g(L), bb(L), twoc2(G);
        for (int l = 0; l < L; ++l) {
            const double z2 = h_r[l] * h_r[l] + h_x[l] * h_x[l];
            g[l] = h_r[l] / z2;                                     // y = 1 / (r + jx)
            bb[l] = -h_x[l] / z2;
        }
        for (int k = 0; k < G; ++k) twoc2[k] = 2.0 * h_c2[k];
        m->from.assign(h_from, h_from + L);
        m->to.assign(h_to, h_to + L);
        m->gen_bus.assign(h_gen_bus, h_gen_bus + G);
        m->c2.assign(h_c2, h_c2 + G);
        if (flags & KKT_MODEL_HOST_ONLY) {
            *out = m;
            return KKT_OK;
        }
        // device copies
        auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
        const size_t sz[] = {al(4 * (size_t)L), al(4 * (size_t)L), al(4 * tptr.size()), al(4 * std::max<size_t>(tidx.size(), 1)),
                             al(4 * kind.size()), al(4 * arg.size()), al(8 * (size_t)L), al(8 * (size_t)L),
                             al(8 * std::max(G, 1)), al(8 * (size_t)L * kLineTerms + 8)};
        size_t total = 0;
        for (size_t v : sz) total += v;
        if (cudaMalloc(&m->base, total) != cudaSuccess) {
            cudaGetLastError();
            delete m;
            return KKT_E_NOMEM;
        }
        char* p = m->base;
        m->d_f = (int*)p; p += sz[0];
        m->d_t = (int*)p; p += sz[1];
        m->d_tptr = (int*)p; p += sz[2];
        m->d_tidx = (int*)p; p += sz[3];
        m->d_kind = (int*)p; p += sz[4];
        m->d_arg = (int*)p; p += sz[5];
        m->d_g = (double*)p; p += sz[6];
        m->d_b = (double*)p; p += sz[7];
        m->d_twoc2 = (double*)p; p += sz[8];
        m->d_terms = (double*)p;
        // through a private non-blocking stream, waited for before returning (a
        // plain cudaMemcpy from pageable memory may return before the device
        // holds the data, unordered with the caller's non-blocking streams)
        cudaStream_t ust = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&ust, cudaStreamNonBlocking);
        auto up = [&](void* d, const void* h, size_t b) {
            if (e == cudaSuccess && b) e = cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, ust);
        };
        up(m->d_f, h_from, 4 * (size_t)L);
        up(m->d_t, h_to, 4 * (size_t)L);
        up(m->d_tptr, tptr.data(), 4 * tptr.size());
        up(m->d_tidx, tidx.data(), 4 * tidx.size());
        up(m->d_kind, kind.data(), 4 * kind.size());
        up(m->d_arg, arg.data(), 4 * arg.size());
        up(m->d_g, g.data(), 8 * (size_t)L);
        up(m->d_b, bb.data(), 8 * (size_t)L);
        up(m->d_twoc2, twoc2.data(), 8 * (size_t)G);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ust);
        if (ust) cudaStreamDestroy(ust);
        if (e != cudaSuccess) {
            kkt_model_destroy(m);
            return KKT_E_CUDA;
        }
    } catch (const std::bad_alloc&) {
        delete m;
        return KKT_E_NOMEM;
    }
    *out = m;
    return KKT_OK;
}

kkt_status kkt_model_pattern(const kkt_model* m, int32_t* n, int32_t* n_primal, int64_t* nnz, int32_t* h_rowptr,
                             int32_t* h_colidx)
{
    if (!m || !n || !n_primal || !nnz) return KKT_E_ARG;
    *n = m->n;
    *n_primal = m->n_primal;
    *nnz = m->nnz;
    if (h_rowptr) std::memcpy(h_rowptr, m->rowptr.data(), sizeof(int32_t) * (m->n + 1));
    if (h_colidx) std::memcpy(h_colidx, m->colidx.data(), sizeof(int32_t) * m->nnz);
    return KKT_OK;
}

kkt_status kkt_model_assemble(const kkt_model* m, const double* d_V, const double* d_theta, const double* d_lambda,
                              const double* d_sigma, const double* d_dual_diag, double delta_w, double delta_c,
                              double* d_vals, void* stream)
{
    if (!m || !d_V || !d_theta || !d_lambda || !d_sigma || !d_vals) return KKT_E_ARG;
    if (!m->base) return KKT_E_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    if (m->nl > 0)
        line_terms_kernel<<<(m->nl + 127) / 128, 128, 0, st>>>(m->nb, m->nl, m->flow, m->d_f, m->d_t, m->d_g, m->d_b,
                                                               d_V, d_theta, d_lambda, m->d_terms);
    const int blocks = (int)((m->nnz + 255) / 256);
    gather_values_kernel<<<blocks, 256, 0, st>>>(m->nnz, m->d_tptr, m->d_tidx, m->d_kind, m->d_arg, m->d_terms,
                                                 d_sigma, d_dual_diag, m->d_twoc2, 2 * m->nb, m->ng, delta_w, delta_c,
                                                 d_vals);
    return cudaGetLastError() == cudaSuccess ? KKT_OK : KKT_E_CUDA;
}

kkt_status kkt_model_destroy(kkt_model* m)
{
    if (!m) return KKT_OK;
    if (m->base) cudaFree(m->base);
    if (m->ipm_base) cudaFree(m->ipm_base);
    if (m->ipm_pin) cudaFreeHost(m->ipm_pin);
    delete m;
    return KKT_OK;
}

}  // extern "C"
