// rk_residual_noalloc: the residual reduction of one implicit step for callers that
// cannot allocate device memory.  Its scratch (per-block partial sums) is a
// file-scope device array of fixed size, shared by every call in the process.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "rykov.h"

namespace {

constexpr int NA_BS = 256;                                    // threads per block
constexpr int NA_MAX_BLOCKS = RK_NOALLOC_MAX_CELLS / NA_BS;   // 4096 blocks
constexpr int NA_MAX_DEVICES = 64;

// Per-block partial sums: 12 doubles per block (|W_new - W_old| per component,
// then the denominators).  Every block of a call writes its own row before the
// final kernel reads it, so nothing has to be cleared between calls; calls that
// overlap on the GPU race on these rows.
static __device__ __align__(256) double g_partials[NA_MAX_BLOCKS * 12];

// device address of g_partials, looked up once per device
double* g_addr[NA_MAX_DEVICES] = {nullptr};
std::mutex g_mu;

thread_local std::string g_err;

int na_fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

__device__ __forceinline__ void block_sum12(double (&v)[12], double* smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NA_BS / 32;
#pragma unroll
    for (int j = 0; j < 12; ++j)
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    if (lane == 0)
        for (int j = 0; j < 12; ++j) smem[j * NW + warp] = v[j];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int j = 0; j < 12; ++j) {
            double t = smem[j * NW];
            for (int q = 1; q < NW; ++q) t += smem[j * NW + q];
            v[j] = t;
        }
}

// per-block partials of sum_i |W_new - W_old| and sum_i |W_old| (momentum rows:
// sum_i |rho U|_i), the residual definition of rk_implicit_iterate
__global__ void __launch_bounds__(NA_BS) k_res_partials(const double* Wn, const double* Wo, int n,
                                                        double* part) {
    __shared__ double red[12 * (NA_BS / 32)];
    const int i = blockIdx.x * NA_BS + threadIdx.x;
    double v[12];
    for (int j = 0; j < 12; ++j) v[j] = 0.0;
    if (i < n) {
        const double* a = Wn + 6 * (size_t)i;
        const double* b = Wo + 6 * (size_t)i;
        for (int m = 0; m < 6; ++m) v[m] = fabs(a[m] - b[m]);
        const double mom = sqrt(b[1] * b[1] + b[2] * b[2] + b[3] * b[3]);
        v[6] = fabs(b[0]); v[7] = mom; v[8] = mom; v[9] = mom; v[10] = fabs(b[4]); v[11] = fabs(b[5]);
    }
    block_sum12(v, red);
    if (threadIdx.x == 0)
        for (int j = 0; j < 12; ++j) part[(size_t)blockIdx.x * 12 + j] = v[j];
}

__global__ void __launch_bounds__(NA_BS) k_res_final(const double* part, int nblocks, double* out) {
    __shared__ double red[12 * (NA_BS / 32)];
    double v[12];
    for (int j = 0; j < 12; ++j) v[j] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += NA_BS)
        for (int j = 0; j < 12; ++j) v[j] += part[(size_t)b * 12 + j];
    block_sum12(v, red);
    if (threadIdx.x == 0)
        for (int m = 0; m < 6; ++m) out[m] = v[m] / (v[6 + m] > 1e-300 ? v[6 + m] : 1e-300);
}

}  // namespace

extern "C" int rk_residual_noalloc(const double* W_new, const double* W_old, int64_t n_cell,
                                   double* res_out, uintptr_t cuda_stream) {
    g_err.clear();                   // the message describes this call only
    if (!W_new || !W_old || !res_out) return na_fail(RK_EINVAL, "rk_residual_noalloc: null pointer");
    if (n_cell <= 0) return na_fail(RK_EINVAL, "rk_residual_noalloc: n_cell must be positive");
    if (n_cell > RK_NOALLOC_MAX_CELLS)
        return na_fail(RK_EINVAL, "rk_residual_noalloc: n_cell " + std::to_string(n_cell) +
                                      " exceeds the fixed maximum " + std::to_string(RK_NOALLOC_MAX_CELLS));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(RK_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(RK_EINVAL, "rk_residual_noalloc: device id out of range");
    double* part = nullptr;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    {
        // look up the array's device address on this device (which is current): the
        // symbol name itself is only a host-side stand-in.  It is looked up again on
        // every call outside stream capture (so a device reset, which reloads the
        // module, cannot leave a stale address); during capture the address of the
        // last uncaptured call on this device is used
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(s, &cs);
        if (e != cudaSuccess) return na_fail(RK_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
        std::lock_guard<std::mutex> lk(g_mu);
        if (cs == cudaStreamCaptureStatusNone) g_addr[dev] = nullptr;
        if (!g_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_partials);
            if (e != cudaSuccess)
                return na_fail(RK_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_addr[dev] = static_cast<double*>(p);
        }
        part = g_addr[dev];
    }
    const int nblocks = (int)((n_cell + NA_BS - 1) / NA_BS);
    k_res_partials<<<nblocks, NA_BS, 0, s>>>(W_new, W_old, (int)n_cell, part);
    k_res_final<<<1, NA_BS, 0, s>>>(part, nblocks, res_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(RK_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return RK_OK;
}

extern "C" const char* rk_noalloc_last_error(void) { return g_err.c_str(); }
