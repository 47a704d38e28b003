// clb_reduce.cuh -- FP64 reductions: mean Nusselt number of a wall (Sec. 3.2)
// and the steady-state residual.  Two-level and fixed-order (block tree of
// warp shuffles -> per-block partials -> one block), so results are
// bit-reproducible run to run.
#pragma once
#include "clb_kernels.cuh"

namespace clb {

constexpr int kRedThreads = 256;
constexpr int kMaxResidualBlocks = 2432;   // 152 SMs x 16 resident 256-thread blocks

// Number of partial slots a handle needs (per reduced quantity).
inline int reduce_partials(int nx, int ny) {
    const long long n = (long long)nx * ny;
    long long nb = (n + kRedThreads - 1) / kRedThreads;
    if (nb > kMaxResidualBlocks) nb = kMaxResidualBlocks;
    const int m = (nx > ny ? nx : ny);
    const long long nw = (m + kRedThreads - 1) / kRedThreads;
    return (int)(nb > nw ? nb : nw);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a block of kRedThreads threads; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = threadIdx.x < (kRedThreads / 32) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) v = warp_sum(v);
    __syncthreads();
    return v;
}

// Temperature (Eq. 36) of node (x, y) at the current time level; wall nodes
// give their wall value or the second-order adiabatic extrapolation.
template <class P>
__device__ __forceinline__ double temperature_at(const BufT<const typename P::S>& B, const AuxT<typename P::R>& A,
                                                 const KParamsT<typename P::R>& K, int x, int y) {
    using R = typename P::R;
    WallInfo w;
    R v[5];
    // a rest-centred form carries T - T0
    const double toff = P::kCentred ? (double)K.T0 : 0.0;
    if (!wall_info(K.g, K.b, x, y, w)) {
        P::pull5(B, A, K, x, y, v);
        return toff + (double)(sum5(v) * K.p.inv_sigma);
    }
    if (w.st >= 0) return (double)K.b.Tw[w.st];
    P::pull5(B, A, K, x + w.dx, y + w.dy, v);
    const R Ts = sum5(v) * K.p.inv_sigma;
    P::pull5(B, A, K, x + 2 * w.dx, y + 2 * w.dy, v);
    const R Tss = sum5(v) * K.p.inv_sigma;
    return toff + (double)((R(4) * Ts - Tss) * R(1.0 / 3.0));
}

// Per-block partial sums of the trapezoid-weighted local Nusselt number
// Nu = -L dT/dn / dT along one wall (FP64); `scale` = -L / (dT (len - 1)).
template <class P>
__global__ void __launch_bounds__(kRedThreads) k_nusselt_partial(const BufT<typename P::S> in,
                                                                 const AuxT<typename P::R> A,
                                                                 const KParamsT<typename P::R> K, int side,
                                                                 double scale, double* __restrict__ partial) {
    __shared__ double sh[kRedThreads / 32];
    const BufT<const typename P::S> B = as_const(in);
    const bool along_y = side == 0 || side == 1;
    const int len = along_y ? K.g.ny : K.g.nx;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < len) {
        double T0, T1, T2, d;
        if (side == 0) {
            T0 = temperature_at<P>(B, A, K, 0, i);
            T1 = temperature_at<P>(B, A, K, 1, i);
            T2 = temperature_at<P>(B, A, K, 2, i);
            d = (-3.0 * T0 + 4.0 * T1 - T2) * 0.5;
        } else if (side == 1) {
            const int e = K.g.nx - 1;
            T0 = temperature_at<P>(B, A, K, e, i);
            T1 = temperature_at<P>(B, A, K, e - 1, i);
            T2 = temperature_at<P>(B, A, K, e - 2, i);
            d = (3.0 * T0 - 4.0 * T1 + T2) * 0.5;
        } else if (side == 2) {
            T0 = temperature_at<P>(B, A, K, i, 0);
            T1 = temperature_at<P>(B, A, K, i, 1);
            T2 = temperature_at<P>(B, A, K, i, 2);
            d = (-3.0 * T0 + 4.0 * T1 - T2) * 0.5;
        } else {
            const int e = K.g.ny - 1;
            T0 = temperature_at<P>(B, A, K, i, e);
            T1 = temperature_at<P>(B, A, K, i, e - 1);
            T2 = temperature_at<P>(B, A, K, i, e - 2);
            d = (3.0 * T0 - 4.0 * T1 + T2) * 0.5;
        }
        const double wgt = (i == 0 || i == len - 1) ? 0.5 : 1.0;
        v = scale * d * wgt;
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

// Residual sums over all nodes: |u - u_ref|^2, |u|^2, (T - T_ref)^2, T^2;
// the reference is replaced by the current fields.  cur/ref hold
// (ux, uy, T) as three consecutive dense fields of n values.
__global__ void __launch_bounds__(kRedThreads) k_residual_partial(const double* __restrict__ cur,
                                                                  double* __restrict__ ref, long long n,
                                                                  double* __restrict__ partial, int nb) {
    __shared__ double sh[kRedThreads / 32];
    double du = 0.0, uu = 0.0, dt = 0.0, tt = 0.0;
    for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kRedThreads) {
        const double a = cur[i], b = cur[n + i], t = cur[2 * n + i];
        const double ea = a - ref[i], eb = b - ref[n + i], et = t - ref[2 * n + i];
        du = fma(ea, ea, fma(eb, eb, du));
        uu = fma(a, a, fma(b, b, uu));
        dt = fma(et, et, dt);
        tt = fma(t, t, tt);
        ref[i] = a;
        ref[n + i] = b;
        ref[2 * n + i] = t;
    }
    du = block_sum(du, sh);
    uu = block_sum(uu, sh);
    dt = block_sum(dt, sh);
    tt = block_sum(tt, sh);
    if (threadIdx.x == 0) {
        partial[0 * nb + blockIdx.x] = du;
        partial[1 * nb + blockIdx.x] = uu;
        partial[2 * nb + blockIdx.x] = dt;
        partial[3 * nb + blockIdx.x] = tt;
    }
}

// result[k] = sum_b partial[k * nb + b], k < nk, in a fixed order.
__global__ void __launch_bounds__(kRedThreads) k_sum_partials(const double* __restrict__ partial, int nb, int nk,
                                                              double* __restrict__ result) {
    __shared__ double sh[kRedThreads / 32];
    for (int k = 0; k < nk; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += kRedThreads) v += partial[k * nb + b];
        v = block_sum(v, sh);
        if (threadIdx.x == 0) result[k] = v;
    }
}

}  // namespace clb
