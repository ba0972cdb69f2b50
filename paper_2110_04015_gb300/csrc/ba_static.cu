// Allocation-free true-residual check: ba_schur_residual_static (declared in include/ba.h).
//
// Some callers cannot allocate device memory at the point where they want to check a
// solution: real-time loops whose memory budget is fixed up front, or hosts whose allocator owns
// all device memory.  This entry point
// computes |-b~ - S x| and |b~| for a block-sparse S the caller already holds on the device,
// without any allocation: its only working memory is the file-scope device array below.
//
// The array is part of the loaded library image, so every GPU that loads the library holds it
// (1 MiB) until the process exits.  Host code cannot use the array's name as a device address;
// the address comes from cudaGetSymbolAddress with the device current.  Outside a stream capture
// it is looked up again on every call, so a call after cudaDeviceReset (which reloads the module)
// or from another context of the device gets the current address; while the call's stream is
// capturing, the address from the last call made outside capture on that device is used.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "ba_internal.cuh"

namespace ba {

namespace {

// per block-row partial sums: [0, BA_STATIC_MAX_CAMS) holds |t_j|^2, the rest |b~_j|^2
static __device__ __align__(256) double g_residual_scratch[2 * BA_STATIC_MAX_CAMS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

// One warp per block-row j: t_j = -b~_j - sum_q S_jq x_col(q) (row-major 9x9 blocks),
// scratch[j] = |t_j|^2, scratch[max + j] = |b~_j|^2.  Every row is written on every call.
__global__ void k_static_rows(int32_t n_c, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                              const double* __restrict__ blocks, const double* __restrict__ bt,
                              const double* __restrict__ x, double* __restrict__ scratch) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t j = w0; j < n_c; j += nw) {
        double acc[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = 0.0;
        for (int64_t q = row_ptr[j] + lane; q < row_ptr[j + 1]; q += 32) {
            const double* B = blocks + q * 81;
            const double* xk = x + int64_t(col[q]) * 9;
            double xv[9];
#pragma unroll
            for (int b = 0; b < 9; ++b) xv[b] = xk[b];
#pragma unroll
            for (int a = 0; a < 9; ++a)
#pragma unroll
                for (int b = 0; b < 9; ++b) acc[a] += B[9 * a + b] * xv[b];
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = warp_sum_d(acc[a]);
        if (lane == 0) {
            double tt = 0.0, bb = 0.0;
            for (int a = 0; a < 9; ++a) {
                const double b = bt[9 * j + a];
                const double t = -b - acc[a];
                tt += t * t;
                bb += b * b;
            }
            scratch[j] = tt;
            scratch[BA_STATIC_MAX_CAMS + j] = bb;
        }
    }
}

// One CTA: out = (sqrt(sum_j scratch[j]), sqrt(sum_j scratch[max + j])), summed in a fixed order.
__global__ void k_static_total(int32_t n_c, const double* __restrict__ scratch, double* __restrict__ out) {
    __shared__ double red[2][256];
    double a = 0.0, b = 0.0;
    for (int j = threadIdx.x; j < n_c; j += blockDim.x) {
        a += scratch[j];
        b += scratch[BA_STATIC_MAX_CAMS + j];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sqrt(red[0][0]);
        out[1] = sqrt(red[1][0]);
    }
}

// Device address of the scratch array on the current device (see the file comment for when it is
// looked up).  A call on a capturing stream with nothing cached yet is refused with STATE.
int scratch_address(cudaStream_t st, double** addr, std::string& err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return BA_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        err = "device index out of range";
        return BA_ERR_INVALID_ARG;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) {
        cudaGetLastError();   // e.g. the legacy stream queried while another stream captures
        cs = cudaStreamCaptureStatusActive;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_residual_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return BA_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    } else if (!g_scratch_addr[dev]) {
        err = "the first call on a device must be made outside a stream capture";
        return BA_ERR_STATE;
    }
    *addr = g_scratch_addr[dev];
    return BA_OK;
}

}  // namespace

}  // namespace ba

extern "C" int ba_schur_residual_static(int32_t n_cams, const int64_t* row_ptr, const int32_t* col,
                                        const double* blocks, const double* btilde, const double* x,
                                        double* out, void* stream) {
    std::string err;
    if (n_cams < 1 || n_cams > BA_STATIC_MAX_CAMS) {
        ba::set_thread_error("ba_schur_residual_static: n_cams must be in [1, " +
                             std::to_string(BA_STATIC_MAX_CAMS) + "], got " + std::to_string(n_cams));
        return BA_ERR_INVALID_ARG;
    }
    if (!row_ptr || !col || !blocks || !btilde || !x || !out) {
        ba::set_thread_error("ba_schur_residual_static: NULL pointer argument");
        return BA_ERR_INVALID_ARG;
    }
    double* scratch = nullptr;
    int code = ba::scratch_address(static_cast<cudaStream_t>(stream), &scratch, err);
    if (code != BA_OK) {
        ba::set_thread_error("ba_schur_residual_static: " + err);
        return code;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int warps_per_cta = ba::kThreads / 32;
    int64_t g = (int64_t(n_cams) + warps_per_cta - 1) / warps_per_cta;
    int cap = ba::num_sms() * 8;
    int grid = int(g < cap ? g : cap);
    ba::k_static_rows<<<grid, ba::kThreads, 0, st>>>(n_cams, row_ptr, col, blocks, btilde, x, scratch);
    ba::k_static_total<<<1, 256, 0, st>>>(n_cams, scratch, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ba::set_thread_error(std::string("ba_schur_residual_static: ") + cudaGetErrorString(e));
        return BA_ERR_CUDA;
    }
    return BA_OK;
}
