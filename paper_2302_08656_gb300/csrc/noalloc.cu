// Allocation-free residual and backward error (kkt_backward_error_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// residual check: a solver embedded in a host framework that owns every byte
// of device memory through its own pool (and forbids foreign allocations), a
// serving loop that must stay inside a fixed memory budget, or code that wants
// to check a solution before any kkt_ctx (and so before any workspace) exists.
// This entry point computes r = b - K x and the normwise backward error
// omega = ||r||_inf / (||K||_inf ||x||_inf + ||b||_inf) with no allocation at
// all: its reduction scratch is a fixed array in device global memory that the
// library declares at file scope, so every GPU that loads the library holds it
// (kNoallocSlots * 4 words = 256 KiB) until the process exits.
//
// Maxima are taken on the bit patterns of |value| as unsigned integers: for
// non-negative doubles that order is the numeric order, and a NaN (exponent
// all ones, mantissa nonzero) sorts above +Inf, so one NaN anywhere in K, x, b
// or r makes omega NaN instead of being dropped as fmax would drop it.
//
// The caller's CSR is checked on the device as it is read: a row whose range
// is not 0 <= rowptr[i] <= rowptr[i+1] <= nnz, or that holds a column index
// outside [0, n), is not read past its bounds; its r_i is set to NaN, and so
// omega comes out NaN.
#include "../../include/kkt.h"

#include <cuda_runtime.h>

#include <math.h>
#include <mutex>

namespace {

constexpr int kRowsPerBlock = 1024;          // 8 warps x 128 rows
constexpr int kNoallocSlots = 8192;          // partial-result slots (one per block)
constexpr int64_t kNoallocMaxRows = (int64_t)kRowsPerBlock * kNoallocSlots;   // 8,388,608

// Shared by every call on a device; each call overwrites the slots it uses.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoallocSlots * 4];

constexpr unsigned kFull = 0xffffffffu;

// |x| as the bits of a non-negative double (NaN above +Inf)
__device__ __forceinline__ unsigned long long mag_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long umax(unsigned long long a, unsigned long long b)
{
    return a > b ? a : b;
}
__device__ __forceinline__ unsigned long long wmax(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) v = umax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ double wsum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Pass 1: one warp per row computes r_i = b_i - sum_j k_ij x_j (lanes stride
// the row, butterfly sum) and the row's |K| sum; every block writes the maxima
// of |r|, |x|, |b| and the K row sums over its rows into its own slot.
__global__ void __launch_bounds__(256) resid_partial_kernel(int n, int64_t nnz, const int* __restrict__ rp,
                                                            const int* __restrict__ ci,
                                                            const double* __restrict__ v,
                                                            const double* __restrict__ x,
                                                            const double* __restrict__ b,
                                                            double* __restrict__ r,
                                                            unsigned long long* scratch)
{
    __shared__ unsigned long long red[4][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int row0 = blockIdx.x * kRowsPerBlock;
    const int row1 = min(n, row0 + kRowsPerBlock);
    unsigned long long mr = 0, mx = 0, mb = 0, mk = 0;
    for (int row = row0 + wid; row < row1; row += 8) {
        const int p0 = rp[row], p1 = rp[row + 1];
        bool bad = p0 < 0 || p1 < p0 || (int64_t)p1 > nnz;
        double s = 0.0, a = 0.0;
        if (!bad) {
            for (int p = p0 + lane; p < p1; p += 32) {
                const int c = ci[p];
                if ((unsigned)c >= (unsigned)n) {      // column outside [0, n): not read
                    bad = true;
                    continue;
                }
                s += v[p] * x[c];
                a += fabs(v[p]);
            }
        }
        bad = __any_sync(kFull, bad);
        s = wsum(s);
        a = wsum(a);
        const double ri = bad ? __longlong_as_double(0x7ff8000000000000ll) : b[row] - s;
        if (lane == 0) r[row] = ri;
        mr = umax(mr, mag_bits(ri));
        mx = umax(mx, mag_bits(x[row]));
        mb = umax(mb, mag_bits(b[row]));
        mk = umax(mk, mag_bits(a));
    }
    if (lane == 0) { red[0][wid] = mr; red[1][wid] = mx; red[2][wid] = mb; red[3][wid] = mk; }
    __syncthreads();
    if (threadIdx.x < 4) {
        unsigned long long m = 0;
        for (int q = 0; q < 8; ++q) m = umax(m, red[threadIdx.x][q]);
        scratch[(int64_t)blockIdx.x * 4 + threadIdx.x] = m;
    }
}

// Pass 2: one warp reduces the slots written by pass 1 and forms omega.
__global__ void omega_final_kernel(int nblk, const unsigned long long* scratch, double* __restrict__ omega)
{
    unsigned long long mr = 0, mx = 0, mb = 0, mk = 0;
    for (int i = threadIdx.x; i < nblk; i += 32) {
        mr = umax(mr, scratch[4 * i + 0]);
        mx = umax(mx, scratch[4 * i + 1]);
        mb = umax(mb, scratch[4 * i + 2]);
        mk = umax(mk, scratch[4 * i + 3]);
    }
    mr = wmax(mr); mx = wmax(mx); mb = wmax(mb); mk = wmax(mk);
    if (threadIdx.x == 0) {
        const double dr = __longlong_as_double((long long)mr), dx = __longlong_as_double((long long)mx);
        const double db = __longlong_as_double((long long)mb), dk = __longlong_as_double((long long)mk);
        const double den = dk * dx + db;
        omega[0] = den > 0.0 ? dr / den : (den == 0.0 ? dr : den);   // a NaN denominator gives NaN
    }
}

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned long long* g_scratch_ptr[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(unsigned long long** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" kkt_status kkt_backward_error_noalloc(int32_t n, int64_t nnz, const int32_t* d_rowptr,
                                                 const int32_t* d_colidx, const double* d_vals,
                                                 const double* d_x, const double* d_rhs, double* d_r,
                                                 double* d_omega, void* stream)
{
    if (n <= 0 || nnz < 0 || !d_rowptr || !d_x || !d_rhs || !d_r || !d_omega) return KKT_E_ARG;
    if (nnz > 0 && (!d_colidx || !d_vals)) return KKT_E_ARG;
    if ((int64_t)n > kNoallocMaxRows) return KKT_E_ARG;   // more rows than the fixed scratch can reduce
    unsigned long long* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return KKT_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int nblk = (int)(((int64_t)n + kRowsPerBlock - 1) / kRowsPerBlock);
    resid_partial_kernel<<<nblk, 256, 0, st>>>(n, nnz, d_rowptr, d_colidx, d_vals, d_x, d_rhs, d_r, scratch);
    omega_final_kernel<<<1, 32, 0, st>>>(nblk, scratch, d_omega);
    return cudaGetLastError() == cudaSuccess ? KKT_OK : KKT_E_CUDA;
}
