// clb_tma.cuh -- the interior of the equilibrium-shifted FP16 step (the
// F16N form) fed by the Tensor Memory Accelerator.
//
// The plain k_step2 has every thread load its pair's 55 source values from
// global memory and hold them in registers while the collision runs; its
// occupancy is set by those registers and the load latency is hidden only
// by the warps resident at the time.  Here a persistent CTA walks tiles of
// TT_X x TT_Y nodes (the rows 1 .. ny - 2, whose sources never wrap) and
// one thread issues, per tile, sixteen bulk tensor copies into a shared
// memory stage:
//   the 9 + 5 distribution planes, each a (TT_X + 16) x TT_Y box starting at
//     (x0 - 8, y0 - e_iy): the rows direction i pulls from (the x start is
//     rounded down to 16 bytes; the x halo of one node lies inside),
//   the record plane (rho - 1, u, T - T0 as halves) and the 1/phi plane,
//     boxes of TT_Y + 2 rows starting at y0 - 1.
// A ring of TT_STAGES stages keeps the next tiles' copies in flight while
// the CTA computes from shared memory; the pull reads each direction's
// values at fixed offsets from the thread's position, the collision and the
// store are those of the plain path (collide_store_pair), so both paths
// produce the same bits.  Edge nodes (first and last pair of a row, walled
// rows) and, for a periodic y, the rows 0 and ny - 1 stay with k_step2.
// The wait on a stage is bounded (`limit` cycles): on expiry the CTA stops,
// waits (with the default bound) for the copies it issued, and sets *fail.
// With `selftest` set, every CTA's first wait is on a barrier that nothing
// completes, which exercises that path without any fault.
#pragma once

#include <cuda.h>

#include "clb_kernels.cuh"

namespace clb {

constexpr int TT_X = 64;                                // nodes per tile row: 32 pairs
constexpr int TT_Y = 4;                                 // rows per tile: 128 pairs, one per thread
constexpr int TT_FX = TT_X + 16;                        // plane box width (x0 - 8 .. x0 + 71)
constexpr int TT_RX = TT_X + 4;                         // record box width (x0 - 2 .. x0 + 65)
constexpr int TT_IX = TT_X + 8;                         // 1/phi box width (x0 - 4 .. x0 + 67)
constexpr int TT_PLANE_B = TT_Y * TT_FX * 2;            // bytes of one plane box (640)
constexpr int TT_R_OFF = 14 * TT_PLANE_B;               // record box offset in a stage
constexpr int TT_R_B = (TT_Y + 2) * TT_RX * 8;          // record box bytes (3264)
constexpr int TT_I_OFF = TT_R_OFF + (TT_R_B + 127) / 128 * 128;
constexpr int TT_I_B = (TT_Y + 2) * TT_IX * 4;          // 1/phi box bytes (1728)
constexpr int TT_STAGE_B = TT_I_OFF + (TT_I_B + 127) / 128 * 128;   // 14080: every box 128-byte aligned
constexpr int TT_TX_BYTES = 14 * TT_PLANE_B + TT_R_B + TT_I_B;      // bytes a stage receives
constexpr int TT_STAGES = 3;
constexpr int TT_THREADS = TT_X / 2 * TT_Y;             // 128: one pair per thread
constexpr int TT_SMEM = TT_STAGES * TT_STAGE_B + 128;   // + alignment slack
constexpr long long TT_LIMIT = 4000000000LL;            // default bound of a wait (~2 s at 2 GHz)
static_assert(TT_THREADS == 128, "one pair per thread");

// e_iy of the nine directions (Eq. 18's lattice, the numbering of sources())
__device__ __forceinline__ constexpr int dir_ey(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__device__ __forceinline__ constexpr int dir_ex(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}

__device__ __forceinline__ uint32_t sm_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void tt_mbar_init(uint32_t a) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
}

__device__ __forceinline__ void tt_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

// Bounded wait for completion `parity` of the mbarrier; false after `limit` SM clock cycles.
__device__ __forceinline__ bool tt_wait(uint32_t a, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tt_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tt_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                           int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// Issue the sixteen copies of tile t into the stage at `dst`.
__device__ __forceinline__ void tt_issue(const CUtensorMap* mf, const CUtensorMap* mg, const CUtensorMap* mr,
                                         const CUtensorMap* mi, uint32_t dst, uint32_t bar, int t, int tiles_x) {
    const int ty = t / tiles_x, x0 = (t - ty * tiles_x) * TT_X, y0 = 1 + ty * TT_Y;
    tt_expect_tx(bar, (uint32_t)TT_TX_BYTES);
#pragma unroll
    for (int i = 0; i < 9; ++i) tt_load_3d(dst + i * TT_PLANE_B, mf, bar, x0 - 8, y0 - dir_ey(i), i);
#pragma unroll
    for (int i = 0; i < 5; ++i) tt_load_3d(dst + (9 + i) * TT_PLANE_B, mg, bar, x0 - 8, y0 - dir_ey(i), i);
    tt_load_2d(dst + TT_R_OFF, mr, bar, x0 - 2, y0 - 1);
    tt_load_2d(dst + TT_I_OFF, mi, bar, x0 - 4, y0 - 1);
}

// Direction I of the pair at tile position (lx, ly), lx even, from the stage.
template <int I>
__device__ __forceinline__ void pull2_tile(const unsigned char* st, int lx, int ly, const KParamsT<float>& K,
                                           f2 (&f)[9], f2 (&g)[5]) {
    constexpr int ex = dir_ex(I), ey = dir_ey(I);
    const uint2* rec = reinterpret_cast<const uint2*>(st + TT_R_OFF) + (ly - ey + 1) * TT_RX + (lx - ex + 2);
    const float* ipp = reinterpret_cast<const float*>(st + TT_I_OFF) + (ly - ey + 1) * TT_IX + (lx - ex + 4);
    const __half* fp = reinterpret_cast<const __half*>(st + I * TT_PLANE_B) + ly * TT_FX + (lx - ex + 8);
    const __half* gp =
        reinterpret_cast<const __half*>(st + (9 + (I < 5 ? I : 0)) * TT_PLANE_B) + ly * TT_FX + (lx - ex + 8);
    uint2 r0, r1;
    float2 ip, df, dg = make_float2(0.0f, 0.0f);
    if (ex == 0) {   // both sources in one aligned vector
        const uint4 r = *reinterpret_cast<const uint4*>(rec);
        r0 = make_uint2(r.x, r.y);
        r1 = make_uint2(r.z, r.w);
        ip = *reinterpret_cast<const float2*>(ipp);
        df = __half22float2(*reinterpret_cast<const __half2*>(fp));
        if (I < 5) dg = __half22float2(*reinterpret_cast<const __half2*>(gp));
    } else {
        r0 = rec[0];
        r1 = rec[1];
        ip = make_float2(ipp[0], ipp[1]);
        df = make_float2(__half2float(fp[0]), __half2float(fp[1]));
        if (I < 5) dg = make_float2(__half2float(gp[0]), __half2float(gp[1]));
    }
    StoreH16NT<LdNC>::combine2<I>(r0, r1, ip, df, dg, K, f, g);
}

// Resident CTAs per SM the kernel is compiled for (shared memory allows five).
#ifndef CLB_TT_MINB
#define CLB_TT_MINB 5
#endif

template <bool SHIFT, bool FORCH>
__global__ void __launch_bounds__(TT_THREADS, CLB_TT_MINB)
    k_step2n_tma(const __grid_constant__ CUtensorMap mf, const __grid_constant__ CUtensorMap mg,
                 const __grid_constant__ CUtensorMap mr, const __grid_constant__ CUtensorMap mi,
                 const BufT<__half> in, const BufT<__half> out, const AuxT<float> A, const KParamsT<float> K,
                 int tiles_x, int ntiles, long long limit, int selftest, unsigned* fail) {
    extern __shared__ unsigned char tt_raw[];
    unsigned char* const sm = tt_raw + ((128u - (sm_u32(tt_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t full[TT_STAGES];
    __shared__ __align__(8) uint64_t dead;   // self-test: a barrier that nothing completes
    __shared__ int s_fail;
    const int tid = threadIdx.x, lx = 2 * (tid & 31), ly = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < TT_STAGES; ++s) tt_mbar_init(sm_u32(&full[s]));
        tt_mbar_init(sm_u32(&dead));
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint32_t seq = in.seq ? __ldg(in.seq) : 0u;
    const PhysT<f2> P2 = splat(K.p);
    int issued = 0;
    if (tid == 0)
        for (int s = 0; s < TT_STAGES; ++s) {
            const int t = blockIdx.x + s * gridDim.x;
            if (t >= ntiles) break;
            tt_issue(&mf, &mg, &mr, &mi, sm_u32(sm + s * TT_STAGE_B), sm_u32(&full[s]), t, tiles_x);
            ++issued;
        }
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int st = k % TT_STAGES;
        const bool dummy = selftest && k == 0;
        if (!tt_wait(sm_u32(dummy ? &dead : &full[st]), dummy ? 0u : (uint32_t)((k / TT_STAGES) & 1), limit))
            s_fail = 1;
        const int ty = t / tiles_x;
        const int x0 = (t - ty * tiles_x) * TT_X + lx, y = 1 + ty * TT_Y + ly;
        if (!s_fail && y <= K.g.ny - 2 && interior_pair(K.g, x0, y)) {
            const unsigned char* stage = sm + st * TT_STAGE_B;
            f2 f[9], g[5];
            pull2_tile<0>(stage, lx, ly, K, f, g);
            pull2_tile<1>(stage, lx, ly, K, f, g);
            pull2_tile<2>(stage, lx, ly, K, f, g);
            pull2_tile<3>(stage, lx, ly, K, f, g);
            pull2_tile<4>(stage, lx, ly, K, f, g);
            pull2_tile<5>(stage, lx, ly, K, f, g);
            pull2_tile<6>(stage, lx, ly, K, f, g);
            pull2_tile<7>(stage, lx, ly, K, f, g);
            pull2_tile<8>(stage, lx, ly, K, f, g);
            const float2 q = *reinterpret_cast<const float2*>(stage + TT_I_OFF + 4 * ((ly + 1) * TT_IX + lx + 4));
            const f2 ip = f2::make(q.x, q.y);
            const CoefT<f2> c = coef2_from_phi<FORCH>(recip(ip), ip, A.ayg[y], K);
            collide_store_pair<StoreH16NT<LdNC>, SHIFT, FORCH>(f, g, c, P2, out, K, x0, y, seq);
        }
        __syncthreads();   // every thread is done with stage st (and has seen s_fail)
        if (s_fail) break;
        if (tid == 0) {
            const int tn = t + TT_STAGES * gridDim.x;
            if (tn < ntiles) {
                tt_issue(&mf, &mg, &mr, &mi, sm_u32(sm + st * TT_STAGE_B), sm_u32(&full[st]), tn, tiles_x);
                ++issued;
            }
        }
    }
    if (s_fail && tid == 0) {
        // copies still in flight write this CTA's shared memory: wait for them (bounded)
        for (int j = k; j < issued; ++j)
            tt_wait(sm_u32(&full[j % TT_STAGES]), (uint32_t)((j / TT_STAGES) & 1), TT_LIMIT);
        atomicExch(fail, 1u);
    }
}

}  // namespace clb
