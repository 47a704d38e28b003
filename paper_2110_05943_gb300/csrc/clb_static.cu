// clb_static.cu -- mean Nusselt number of a wall from a caller-provided
// device temperature field, without allocating any memory.
//
// The per-block partial sums live in a fixed array in this file's device
// memory instead of a buffer obtained from cudaMalloc.  Host code cannot use
// the array's name as a device address, so the address is looked up with
// cudaGetSymbolAddress (which allocates nothing), with the device current.
// A call made outside stream capture looks it up afresh -- after a
// cudaDeviceReset or under another context of the same device the array
// lives at a new address -- and caches it per device; a call made while its
// stream is being captured uses that cache, because the lookup may have to
// load the module, which capture does not allow.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/clb.h"

void clb_internal_set_error(const char* msg);   // defined in clb_api.cu

namespace {

constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// Block partials of the reduction; every call overwrites the slots it reads,
// so nothing has to be cleared between calls.
__device__ __align__(256) double s_partials[CLB_STATIC_MAX_PARTIALS];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
    if (wid == 0) v = warp_sum(v);
    return v;
}

// One thread per node along the wall: trapezoid-weighted local
// Nu = -L dT/dn / dT from the one-sided second-order difference.
__global__ void __launch_bounds__(kThreads) k_nu_field_partial(const double* __restrict__ T, int nx, int ny,
                                                               int side, double scale, double* __restrict__ part) {
    const bool along_y = side == CLB_W || side == CLB_E;
    const int len = along_y ? ny : nx;
    const int i = blockIdx.x * kThreads + threadIdx.x;
    double v = 0.0;
    if (i < len) {
        const long long r = (long long)i * nx;
        double d;
        if (side == CLB_W)
            d = (-3.0 * T[r] + 4.0 * T[r + 1] - T[r + 2]) * 0.5;
        else if (side == CLB_E)
            d = (3.0 * T[r + nx - 1] - 4.0 * T[r + nx - 2] + T[r + nx - 3]) * 0.5;
        else if (side == CLB_S)
            d = (-3.0 * T[i] + 4.0 * T[nx + i] - T[2LL * nx + i]) * 0.5;
        else {
            const long long e = (long long)(ny - 1) * nx + i;
            d = (3.0 * T[e] - 4.0 * T[e - nx] + T[e - 2LL * nx]) * 0.5;
        }
        v = scale * d * ((i == 0 || i == len - 1) ? 0.5 : 1.0);
    }
    v = block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kThreads) k_nu_field_sum(const double* __restrict__ part, int nb,
                                                           double* __restrict__ out) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += kThreads) v += part[b];
    v = block_sum(v);
    if (threadIdx.x == 0) *out = v;
}

int fail(int code, const char* msg) {
    clb_internal_set_error(msg);
    return code;
}

// Device address of s_partials in the current context: looked up afresh
// unless the stream is being captured, then taken from the per-device cache.
int scratch_address(cudaStream_t stream, double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(CLB_ERR_CUDA, "clb_nusselt_field_static: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return fail(CLB_ERR_ARG, "clb_nusselt_field_static: device index too large");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess)
        return fail(CLB_ERR_CUDA, "clb_nusselt_field_static: cudaStreamIsCapturing failed");
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap != cudaStreamCaptureStatusNone) {
        if (!g_addr[dev])
            return fail(CLB_ERR_ARG,
                        "clb_nusselt_field_static: first call on this device made during stream capture; "
                        "call it once before capturing");
    } else {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, s_partials);
        if (e != cudaSuccess || !p) {
            char buf[256];
            std::snprintf(buf, sizeof buf, "clb_nusselt_field_static: cudaGetSymbolAddress failed: %s",
                          cudaGetErrorString(e));
            return fail(CLB_ERR_CUDA, buf);
        }
        g_addr[dev] = (double*)p;
    }
    *out = g_addr[dev];
    return CLB_OK;
}

}  // namespace

extern "C" int clb_nusselt_field_static(const double* T, int32_t nx, int32_t ny, int32_t side, double L, double dT,
                                        double* nu, void* stream) {
    if (!T || !nu) return fail(CLB_ERR_ARG, "clb_nusselt_field_static: T and nu must be device pointers");
    if (side < 0 || side > 3) return fail(CLB_ERR_ARG, "clb_nusselt_field_static: side must be 0..3");
    const bool along_y = side == CLB_W || side == CLB_E;
    const long long len = along_y ? ny : nx, depth = along_y ? nx : ny;
    if (len < 2 || depth < 3) return fail(CLB_ERR_ARG, "clb_nusselt_field_static: grid too small");
    if (!(L > 0) || !(dT > 0) || !std::isfinite(L) || !std::isfinite(dT))
        return fail(CLB_ERR_ARG, "clb_nusselt_field_static: L and dT must be positive");
    const long long nb = (len + kThreads - 1) / kThreads;
    if (nb > CLB_STATIC_MAX_PARTIALS)
        return fail(CLB_ERR_ARG, "clb_nusselt_field_static: wall longer than CLB_STATIC_MAX_WALL nodes");
    // an error left by earlier, unrelated work is reported as such and left
    // in place for its owner (cudaGetLastError below would clear it)
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "clb_nusselt_field_static: a CUDA error was pending before the call: %s",
                      cudaGetErrorString(pending));
        return fail(CLB_ERR_CUDA, buf);
    }
    cudaStream_t s = (cudaStream_t)stream;
    double* part = nullptr;
    const int rc = scratch_address(s, &part);
    if (rc != CLB_OK) return rc;
    const double scale = -L / dT / (double)(len - 1);
    k_nu_field_partial<<<(unsigned)nb, kThreads, 0, s>>>(T, nx, ny, side, scale, part);
    k_nu_field_sum<<<1, kThreads, 0, s>>>(part, (int)nb, nu);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "clb_nusselt_field_static: launch failed: %s", cudaGetErrorString(e));
        return fail(CLB_ERR_CUDA, buf);
    }
    return CLB_OK;
}
