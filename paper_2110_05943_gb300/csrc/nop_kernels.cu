// nop_kernels.cu -- kernels of the learned warm start: a small convolutional
// neural operator (U-Net-like) that maps (porosity field, Ra, Da, Pr, sigma)
// to the steady (u, v, T) of the porous cavity, trained on steady states the
// LB solver generates.  BF16 weights and activations, FP32 accumulation.
//
// Layout: activations NHWC (channels fastest), BF16.  Convolution weights
// as a [taps * Cin][Cout] matrix (Cout fastest), taps = 9 (3x3) or 1 (1x1).
// Every convolution pass is an implicit GEMM on the BF16 tensor cores with
// FP32 accumulation:
//   forward : Y[p, co]   = sum_{tap, ci} X[p + d(tap), ci] W[tap, ci, co] (+ b, ReLU)
//   dgrad   : dX[p, ci]  = sum_{tap, co} dY[p - d(tap), co] W[tap, ci, co]
//   wgrad   : dW[tap, ci, co] += sum_p X[p + d(tap), ci] dY[p, co]   (split K, FP32 atomics)
// In order of preference (the first that takes the shape runs):
//   k_conv_tma / k_wgrad_tma -- operands brought by TMA from the NHWC tensors
//     into swizzled shared memory, tcgen05.mma with the accumulator in TMEM
//     (whole-row pixel tiles, channel counts multiples of 8);
//   k_conv_tc / k_wgrad_tc   -- the same MMAs with operands gathered by all
//     threads through registers (any width);
//   k_wgrad_small / k_dgrad_small -- CUDA cores, the 1x1 head (4 outputs);
//   k_conv_gemm              -- mma.sync m16n8k16, 64 x 64 output tiles,
//     operands gathered with zero fill at image borders and tile tails (any
//     channel count).
#include <cuda.h>           // CUtensorMap and its enums (the encoder is fetched at run time)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>   // PFN_cuTensorMapEncodeTiled
#include <stdint.h>

#include <algorithm>

#include "../../include/clb_nop.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;
constexpr int kThreads = 128;

enum Mode { FWD = 0, DGRAD = 1, WGRAD = 2 };

struct ConvShape {
    int n, h, w, cin, cout, taps;   // taps = 9 (3x3, padding 1) or 1 (1x1)
};

__device__ __forceinline__ int tap_dy(int t, int taps) { return taps == 9 ? t / 3 - 1 : 0; }
__device__ __forceinline__ int tap_dx(int t, int taps) { return taps == 9 ? t % 3 - 1 : 0; }

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One 64 x 64 output tile over the K range [kb, kb + kchunk).  Index
// arithmetic is 32-bit (the host rejects larger tensors).  The 64 rows' pixel
// (FWD, DGRAD) or (tap, channel) (WGRAD) decompositions are computed once per
// block; each thread keeps one K column (tid % 32) of both tiles, so its K
// decomposition is computed once per chunk.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_conv_gemm(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
                                                        const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask,
                                                        void* __restrict__ out, int out_f32, int relu, ConvShape s,
                                                        int M, int N, int K, int kchunk) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];   // stored [n][k]
    __shared__ int rb[BM], ry[BM], rx[BM];                      // per-row base / offsets, ry < -2 marks an empty row
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kb = blockIdx.z * kchunk;
    const int ke = kb + kchunk < K ? kb + kchunk : K;
    const int hw = s.h * s.w;
    if (tid < BM) {
        const int m = m0 + tid;
        if (m >= M) {
            rb[tid] = 0; ry[tid] = -1000000; rx[tid] = 0;
        } else if (MODE != WGRAD) {
            const int n = m / hw, rem = m - n * hw, y = rem / s.w;
            rb[tid] = n * s.h; ry[tid] = y; rx[tid] = rem - y * s.w;
        } else {
            const int tap = m / s.cin;
            rb[tid] = m - tap * s.cin; ry[tid] = tap_dy(tap, s.taps); rx[tid] = tap_dx(tap, s.taps);
        }
    }
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;
    const int g = lane >> 2, tg = lane & 3;
    const int col = tid & 31, row0 = tid >> 5;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    __syncthreads();
    for (int k0 = kb; k0 < ke; k0 += BK) {
        const int kk = k0 + col;
        const bool kv = kk < ke;
        if (MODE != WGRAD) {
            // A = activations gathered at the tap's shift: k = tap * C + c
            const int C = MODE == FWD ? s.cin : s.cout;
            const int tap = kv ? kk / C : 0, c = kk - tap * C;
            const int sg = MODE == FWD ? 1 : -1;
            const int ddy = sg * tap_dy(tap, s.taps), ddx = sg * tap_dx(tap, s.taps);
#pragma unroll 4
            for (int j = 0; j < BM / 4; ++j) {
                const int r = row0 + 4 * j;
                const int yy = ry[r] + ddy, xx = rx[r] + ddx;
                __nv_bfloat16 v = zero;
                if (kv && yy >= 0 && yy < s.h && xx >= 0 && xx < s.w) v = A[((rb[r] + yy) * s.w + xx) * C + c];
                As[r][col] = v;
            }
            // B = weights; FWD: W[k][n], DGRAD: W[tap * cin + n][co] with k = tap * cout + co
            const int t2 = MODE == DGRAD && kv ? kk / s.cout : 0, co = kk - t2 * s.cout;
#pragma unroll 4
            for (int j = 0; j < BN / 4; ++j) {
                const int nn = row0 + 4 * j, n = n0 + nn;
                __nv_bfloat16 v = zero;
                if (kv && n < N) v = MODE == FWD ? B[kk * s.cout + n] : B[(t2 * s.cin + n) * s.cout + co];
                Bs[nn][col] = v;
            }
        } else {
            // k = pixel: A = X at the row's tap shift, channel rb[r]; B = dY[pixel][n]
            const int n = kv ? kk / hw : 0, rem = kk - n * hw, y = rem / s.w, x = rem - (rem / s.w) * s.w;
#pragma unroll 4
            for (int j = 0; j < BM / 4; ++j) {
                const int r = row0 + 4 * j;
                const int yy = y + ry[r], xx = x + rx[r];
                __nv_bfloat16 v = zero;
                if (kv && yy >= 0 && yy < s.h && xx >= 0 && xx < s.w) v = A[((n * s.h + yy) * s.w + xx) * s.cin + rb[r]];
                As[r][col] = v;
            }
#pragma unroll 4
            for (int j = 0; j < BN / 4; ++j) {
                const int nn = row0 + 4 * j, c = n0 + nn;
                Bs[nn][col] = kv && c < N ? B[kk * s.cout + c] : zero;
            }
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + g;
                af[i][0] = ld_pair(&As[r][ks + tg * 2]);
                af[i][1] = ld_pair(&As[r + 8][ks + tg * 2]);
                af[i][2] = ld_pair(&As[r][ks + tg * 2 + 8]);
                af[i][3] = ld_pair(&As[r + 8][ks + tg * 2 + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8 + g;
                bf[j][0] = ld_pair(&Bs[c][ks + tg * 2]);
                bf[j][1] = ld_pair(&Bs[c][ks + tg * 2 + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }
    // epilogue: element (row, col) of each 16 x 8 accumulator tile
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = m0 + wm + i * 16 + g + (r >= 2 ? 8 : 0);
                const int cc = n0 + wn + j * 8 + tg * 2 + (r & 1);
                if (row >= M || cc >= N) continue;
                float v = acc[i][j][r];
                const int o = row * N + cc;
                if (MODE == WGRAD) {
                    atomicAdd(reinterpret_cast<float*>(out) + o, v);
                    continue;
                }
                if (bias) v += bias[cc];
                if (relu) v = v > 0.0f ? v : 0.0f;
                if (mask && !(__bfloat162float(mask[o]) > 0.0f)) v = 0.0f;
                if (out_f32) reinterpret_cast<float*>(out)[o] = v;
                else reinterpret_cast<__nv_bfloat16*>(out)[o] = __float2bfloat16(v);
            }
}

template <int MODE>
int launch_gemm(const void* A, const void* B, const float* bias, const void* mask, void* out, int out_f32, int relu,
                ConvShape s, long long M, long long N, long long K, int splitk, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0) return CLB_NOP_ERR_ARG;
    // every element index of every operand must fit in 32 bits
    const long long npix = (long long)s.n * s.h * s.w;
    const long long cmax = s.cin > s.cout ? s.cin : s.cout;
    if (npix * cmax * s.taps >= 2147483647LL || M * N >= 2147483647LL) return CLB_NOP_ERR_ARG;
    const long long gm = (M + BM - 1) / BM, gn = (N + BN - 1) / BN;
    if (gn > 65535) return CLB_NOP_ERR_ARG;
    if (splitk < 1) splitk = (int)std::max(1LL, std::min(64LL, K / 4096));   // automatic (weight gradient)
    long long kchunk = (K + splitk - 1) / splitk;
    kchunk = (kchunk + BK - 1) / BK * BK;
    const long long gz = (K + kchunk - 1) / kchunk;
    if (gz > 65535) return CLB_NOP_ERR_ARG;
    k_conv_gemm<MODE><<<dim3((unsigned)gm, (unsigned)gn, (unsigned)gz), kThreads, 0, st>>>(
        (const __nv_bfloat16*)A, (const __nv_bfloat16*)B, bias, (const __nv_bfloat16*)mask, out, out_f32, relu, s,
        (int)M, (int)N, (int)K, (int)kchunk);
    return cudaGetLastError() == cudaSuccess ? CLB_NOP_OK : CLB_NOP_ERR_CUDA;
}

bool bad_shape(int n, int h, int w, int cin, int cout, int taps) {
    return n < 1 || h < 1 || w < 1 || cin < 1 || cout < 1 || (taps != 1 && taps != 9);
}

// ---------------------------------------------------------------- tcgen05 path
// Forward and input-gradient convolutions on the 5th-generation tensor cores
// when the gathered operand's channel count is a multiple of 8 (so 8
// consecutive K indices are 8 contiguous channels of one tap: one 16-byte
// vector).  One CTA per 128-pixel x tile_n output tile; 64-deep K chunks are
// gathered by all 128 threads into double-buffered shared memory in the
// canonical K-major layout without swizzle (8-row x 16-byte core matrices,
// 128 B apart along K and 16 * TC_K B apart along M/N); thread 0 issues four
// tcgen05.mma (M 128, N tile_n, K 16, BF16 x BF16 -> FP32) per chunk and
// commits them to the buffer's mbarrier; the FP32 accumulator lives in TMEM
// and each warp reads its 32 lanes back with tcgen05.ld for the epilogue.
// TC_K: K depth of one staged chunk.  Measured per training batch (all 3x3
// layers, forward + both gradients): 32 -> 3.00 ms, 64 -> 2.78 ms, 128 -> 3.21 ms.
constexpr int TC_M = 128, TC_K = 64, TC_THREADS = 128;
constexpr int TC_KV = TC_K / 8;                              // 16-byte K vectors per row and chunk
constexpr int TC_ROWS8 = TC_K * 16;                          // bytes of 8 rows (K-major stride byte offset)
constexpr int TC_PIX_STEP = TC_THREADS / TC_K;               // weight gradient: threads per chunk pixel
constexpr int TC_A_BYTES = TC_M * TC_K * 2;                  // one A buffer
constexpr long long TC_TIMEOUT_CYCLES = 4000000000LL;        // ~2 s at 2 GHz

__device__ unsigned int g_nop_timeout = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t tc_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t a) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
}

// Waits for completion `parity` of the mbarrier; false after `limit` SM
// clock cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, long long limit = TC_TIMEOUT_CYCLES) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred P;\n mbarrier.test_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tc_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
}

// MODE FWD: A = activations X (C = cin), B = W^T [cout][taps * cin].
// MODE DGRAD: A = output gradient dY (C = cout), B = W [taps * cin][cout]
// read as B^T[ci][tap * cout + co].
template <int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tc(const __nv_bfloat16* __restrict__ A,
                                                        const __nv_bfloat16* __restrict__ B,
                                                        const float* __restrict__ bias,
                                                        const __nv_bfloat16* __restrict__ mask, void* __restrict__ out,
                                                        int out_f32, int relu, ConvShape s, int M, int N, int K,
                                                        int tile_n, int tmem_cols, int vec_out) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int b_bytes = tile_n * TC_K * 2;
    unsigned char* const a_base = smem;                       // two A buffers, TC_A_BYTES apart
    unsigned char* const b_base = smem + 2 * TC_A_BYTES;      // two B buffers, b_bytes apart
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * TC_A_BYTES + 2 * b_bytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * tile_n;
    const int nt = min(tile_n, N - n0);                 // live columns of this tile
    const int ntp = (nt + 15) & ~15;                    // MMA N (multiple of 16)
    const int C = MODE == FWD ? s.cin : s.cout;
    const int sg = MODE == FWD ? 1 : -1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]));
        mbar_init(smem_u32(&mbar[1]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // this thread's A row: pixel m0 + tid
    const int m = m0 + tid;
    int rb = 0, ry = -1000000, rx = 0;
    if (m < M) {
        const int hw = s.h * s.w, n = m / hw, rem = m - n * hw;
        ry = rem / s.w;
        rx = rem - ry * s.w;
        rb = n * s.h;
    }
    const uint32_t idesc = tc_idesc(ntp);
    const int nchunks = (K + TC_K - 1) / TC_K;
    // A row tid of chunk c: TC_KV 16-byte K vectors, loaded one chunk ahead
    // into registers so their latency overlaps the barrier, the MMAs and the
    // next wait
    uint4 va[TC_KV];
    auto load_a = [&](int c) {
#pragma unroll
        for (int kv = 0; kv < TC_KV; ++kv) {
            const int k = c * TC_K + 8 * kv;
            va[kv] = make_uint4(0u, 0u, 0u, 0u);
            if (k < K) {
                const int tap = k / C, ch = k - tap * C;
                const int yy = ry + sg * tap_dy(tap, s.taps), xx = rx + sg * tap_dx(tap, s.taps);
                if (yy >= 0 && yy < s.h && xx >= 0 && xx < s.w)
                    va[kv] = __ldg(reinterpret_cast<const uint4*>(A + ((rb + yy) * s.w + xx) * C + ch));
            }
        }
    };
    load_a(0);
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
        const int bi = c & 1;
        if (c >= 2 && ok) ok = mbar_wait(smem_u32(&mbar[bi]), ((c - 2) >> 1) & 1);
        const int k0 = c * TC_K;
#pragma unroll
        for (int kv = 0; kv < TC_KV; ++kv)
            *reinterpret_cast<uint4*>(a_base + bi * TC_A_BYTES + (tid >> 3) * TC_ROWS8 + kv * 128 + (tid & 7) * 16) =
                va[kv];
        // B: ntp rows, eight 16-byte K vectors each
        for (int e = tid; e < ntp * TC_KV; e += TC_THREADS) {
            const int r = e % ntp, kv = e / ntp, k = k0 + 8 * kv, gn = n0 + r;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (r < nt && k < K) {
                if (MODE == FWD) {
                    v = __ldg(reinterpret_cast<const uint4*>(B + gn * K + k));
                } else {
                    const int tap = k / s.cout, co = k - tap * s.cout;
                    v = __ldg(reinterpret_cast<const uint4*>(B + (tap * s.cin + gn) * s.cout + co));
                }
            }
            *reinterpret_cast<uint4*>(b_base + bi * b_bytes + (r >> 3) * TC_ROWS8 + kv * 128 + (r & 7) * 16) = v;
        }
        if (c + 1 < nchunks) load_a(c + 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(a_base + bi * TC_A_BYTES), b0 = smem_u32(b_base + bi * b_bytes);
#pragma unroll
            for (int ks = 0; ks < TC_K / 16; ++ks)
                tc_mma(tmem, tc_desc(a0 + ks * 256, 128, TC_ROWS8), tc_desc(b0 + ks * 256, 128, TC_ROWS8), idesc,
                       (c > 0 || ks > 0) ? 1u : 0u);
            tc_commit(smem_u32(&mbar[bi]));
        }
    }
    // every thread waits for the last commit (it covers all earlier MMAs)
    if (ok) ok = mbar_wait(smem_u32(&mbar[(nchunks - 1) & 1]), ((nchunks - 1) >> 1) & 1);
    // a thread that timed out earlier skipped its waits but not the barriers;
    // agree on the outcome before touching TMEM
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < ntp; c0 += 8) {
            uint32_t r[8];
            tc_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (row < M) {
                const int o = row * N + n0 + c0;
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    v[j] = __uint_as_float(r[j]);
                    if (bias && c0 + j < nt) v[j] += bias[n0 + c0 + j];
                    if (relu) v[j] = v[j] > 0.0f ? v[j] : 0.0f;
                }
                if (c0 + 8 <= nt && vec_out) {
                    // eight consecutive outputs of this row: one 16-byte (BF16) or two (FP32) stores
                    if (mask) {
                        const uint4 mk = *reinterpret_cast<const uint4*>(mask + o);
                        const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&mk);
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (!(__bfloat162float(mb[j]) > 0.0f)) v[j] = 0.0f;
                    }
                    if (out_f32) {
                        float4* d = reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + o);
                        d[0] = make_float4(v[0], v[1], v[2], v[3]);
                        d[1] = make_float4(v[4], v[5], v[6], v[7]);
                    } else {
                        uint4 pk;
                        __nv_bfloat162* h2 = reinterpret_cast<__nv_bfloat162*>(&pk);
#pragma unroll
                        for (int j = 0; j < 4; ++j) h2[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                        *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(out) + o) = pk;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (c0 + j >= nt) break;
                        float x = v[j];
                        if (mask && !(__bfloat162float(mask[o + j]) > 0.0f)) x = 0.0f;
                        if (out_f32) reinterpret_cast<float*>(out)[o + j] = x;
                        else reinterpret_cast<__nv_bfloat16*>(out)[o + j] = __float2bfloat16(x);
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(&g_nop_timeout, 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}


// ---------------------------------------------------------------- TMA + tcgen05
// Forward and input-gradient convolutions with operands fetched by the Tensor
// Memory Accelerator, in a persistent warp-specialised kernel.  A tile is 128
// pixels = whole image rows (wbox x hbox, wbox * hbox = 128) by tile_n
// outputs; each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// The K loop of a tile runs over (tap, kc-channel chunk), kc = 32 or 64: per
// iteration one 4-D TMA load brings the activations of the tile shifted by
// the tap -- (c0 .. c0 + kc - 1, w0 + dx, h0 + dy, image) -- and the hardware
// fills everything outside the tensor with zeros, which is exactly the
// convolution's zero padding (and pads a chunk past the last channel); one
// 3-D TMA load brings the matching weights, tile_n rows of kc channels.  Both
// land in shared memory as 2 kc-byte rows with the matching swizzle (64 or
// 128 bytes), the K-major layout tcgen05.mma reads (K = 16 per MMA: the
// descriptor start advances 32 bytes).
//   warp 4 (one thread): producer -- a ring of `stages` buffers; each stage's
//     "full" mbarrier expects the bytes of both boxes;
//   warp 5 (one thread): MMA issuer -- kc / 16 MMAs per stage, committed to
//     the stage's "empty" mbarrier; the tile's accumulator alternates between
//     two TMEM buffers, committed to that buffer's "acc_full" mbarrier;
//   warps 0-3: epilogue -- warp w reads TMEM lanes 32w .. 32w + 31 (one pixel
//     per thread) of the finished buffer, adds the bias, applies ReLU or the
//     mask, stores, and releases the buffer ("acc_empty", 128 arrivals), so
//     the next tile's MMAs overlap this tile's epilogue.
// Every wait is bounded; on expiry a role stops, the CTA waits (bounded) for
// the loads and MMAs it issued, frees its TMEM and sets the flag.
constexpr int TM_THREADS = 192;
// Most stages of the copy rings (build-time options).  Shallower rings leave
// shared memory for the weight gradients, which run concurrently on a side
// stream during training: 5 and 3 measured 1.28 ms per training step against
// 1.30 with 8 and 6.
#ifndef CLB_TM_MAX_STAGES
#define CLB_TM_MAX_STAGES 5
#endif
#ifndef CLB_WG_MAX_STAGES
#define CLB_WG_MAX_STAGES 3
#endif
constexpr int TM_BIAS_MAX = 1024;                // outputs whose bias is staged in shared memory

__device__ __forceinline__ void mbar_init_n(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t mbar, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t mbar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Bounded wait with mbarrier.try_wait (the hardware may suspend the thread
// between tries, so idle threads cost little issue bandwidth).
__device__ __forceinline__ bool mbar_wait_try(uint32_t a, uint32_t parity, long long limit) {
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

// Shared-memory descriptor of a K-major operand stored as R-byte rows with
// the R-byte swizzle (R = 128 or 64): 8-row groups 8R bytes apart (stride
// byte offset), descriptor version 1, swizzle mode 2 (128-byte) or 4 (64-byte).
__device__ __forceinline__ uint64_t tc_desc_sw(uint32_t addr, int row_bytes) {
    const uint64_t mode = row_bytes == 128 ? 2ull : 4ull;
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((8 * row_bytes) >> 4) << 32) |
           (1ull << 46) | (mode << 61);
}

// 32 consecutive accumulator columns of this thread's TMEM lane (no wait).
__device__ __forceinline__ void tc_ld32_nowait(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Epilogue of 8 accumulator values of a row: columns c0 .. c0 + 7 of the
// tile (output o = row * N + n0 + c0), bias from shared memory (sb: the
// tile's first column), ReLU, mask, BF16 or FP32 store.
__device__ __forceinline__ void tm_store8(const uint32_t* r, int o, int c0, int nt, const float* sb,
                                          const __nv_bfloat16* __restrict__ mask, void* __restrict__ out,
                                          int out_f32, int relu, int vec_out) {
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        v[j] = __uint_as_float(r[j]);
        if (sb && c0 + j < nt) v[j] += sb[c0 + j];
        if (relu) v[j] = v[j] > 0.0f ? v[j] : 0.0f;
    }
    if (c0 + 8 <= nt && vec_out) {
        if (mask) {
            const uint4 mk = *reinterpret_cast<const uint4*>(mask + o);
            const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&mk);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (!(__bfloat162float(mb[j]) > 0.0f)) v[j] = 0.0f;
        }
        if (out_f32) {
            float4* d = reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + o);
            d[0] = make_float4(v[0], v[1], v[2], v[3]);
            d[1] = make_float4(v[4], v[5], v[6], v[7]);
        } else {
            uint4 pk;
            __nv_bfloat162* h2 = reinterpret_cast<__nv_bfloat162*>(&pk);
#pragma unroll
            for (int j = 0; j < 4; ++j) h2[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
            *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(out) + o) = pk;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (c0 + j >= nt) break;
            float x = v[j];
            if (mask && !(__bfloat162float(mask[o + j]) > 0.0f)) x = 0.0f;
            if (out_f32) reinterpret_cast<float*>(out)[o + j] = x;
            else reinterpret_cast<__nv_bfloat16*>(out)[o + j] = __float2bfloat16(x);
        }
    }
}

// Epilogue of one accumulator row (pixel `row`, outputs n0 .. n0 + nt - 1):
// 32 columns per TMEM load and wait, then the rest 8 at a time.
__device__ __forceinline__ void tm_store_row(uint32_t taddr, int row, int n0, int nt, int tile_n, int N,
                                             const float* sb, const __nv_bfloat16* __restrict__ mask,
                                             void* __restrict__ out, int out_f32, int relu, int vec_out) {
    const int o = row * N + n0;
    int c0 = 0;
    for (; c0 + 32 <= tile_n; c0 += 32) {
        uint32_t r[32];
        tc_ld32_nowait(taddr + (uint32_t)c0, r);
        tc_wait_ld();
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (c0 + 8 * q < nt) tm_store8(r + 8 * q, o + c0 + 8 * q, c0 + 8 * q, nt, sb, mask, out, out_f32, relu, vec_out);
    }
    for (; c0 < tile_n; c0 += 8) {
        uint32_t r[8];
        tc_ld8(taddr + (uint32_t)c0, r);
        if (c0 < nt) tm_store8(r, o + c0, c0, nt, sb, mask, out, out_f32, relu, vec_out);
    }
}

// MODE FWD: A = activations X (C = cin), B = W^T [cout][taps * cin] viewed as
// (cin, taps, cout).  MODE DGRAD: A = output gradient dY (C = cout) at the
// mirrored taps, B = W [taps * cin][cout] viewed as (cout, cin, taps).
// tmem_cols: columns of one accumulator buffer (two are allocated).
template <int MODE>
__global__ void __launch_bounds__(TM_THREADS, 1) k_conv_tma(const __grid_constant__ CUtensorMap mapA,
                                                         const __grid_constant__ CUtensorMap mapB,
                                                         const float* __restrict__ bias,
                                                         const __nv_bfloat16* __restrict__ mask, void* __restrict__ out,
                                                         int out_f32, int relu, ConvShape s, int M, int N, int tile_n,
                                                         int tmem_cols, int vec_out, int stages, int cchunks, int kc,
                                                         int ntiles, int ntn) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* const smem =
        smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);   // swizzled tiles start on 1024 B
    __shared__ float s_bias[TM_BIAS_MAX];                               // the bias of all N outputs
    const int a_bytes = TC_M * kc * 2, b_bytes = tile_n * kc * 2;
    const int stage_bytes = a_bytes + b_bytes;                           // a multiple of 1024 (tile_n % 16 == 0)
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + stages * stage_bytes);
    uint64_t* empty = full + stages;
    uint64_t* acc_full = empty + stages;                                 // [2]
    uint64_t* acc_empty = acc_full + 2;                                  // [2]
    uint64_t* done = acc_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int s_issued, s_consumed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int sg = MODE == FWD ? 1 : -1;
    const int niter = s.taps * cchunks;
    const int hw = s.h * s.w;

    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < stages; ++i) {
            mbar_init(smem_u32(&full[i]));
            mbar_init(smem_u32(&empty[i]));
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]));
            mbar_init_n(smem_u32(&acc_empty[b]), 128);
        }
        mbar_init(smem_u32(done));
        s_issued = 0;
        s_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const bool sbias = bias && N <= TM_BIAS_MAX;
    if (sbias)
        for (int i = tid; i < N; i += TM_THREADS) s_bias[i] = bias[i];
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    bool ok = true;
    if (warp == 4) {
        if (lane == 0) {   // producer
            int it = 0, st = 0, ph = 0;   // global iteration, its stage and the stage's use count parity
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int m0 = (t / ntn) * TC_M, n0 = (t % ntn) * tile_n;
                const int img = m0 / hw, rem = m0 - img * hw, h0 = rem / s.w, w0 = rem - h0 * s.w;
                for (int j = 0; j < niter; ++j) {
                    if (it >= stages && !mbar_wait_try(smem_u32(&empty[st]), ph ^ 1, TC_TIMEOUT_CYCLES)) {
                        ok = false;
                        break;
                    }
                    const int tap = j / cchunks, c0 = (j - tap * cchunks) * kc;
                    const int ddy = sg * tap_dy(tap, s.taps), ddx = sg * tap_dx(tap, s.taps);
                    const uint32_t fb = smem_u32(&full[st]), a_dst = smem_u32(smem + st * stage_bytes);
                    mbar_expect_tx(fb, (uint32_t)stage_bytes);
                    tma_load_4d(a_dst, &mapA, fb, c0, w0 + ddx, h0 + ddy, img);
                    if (MODE == FWD) tma_load_3d(a_dst + a_bytes, &mapB, fb, c0, tap, n0);
                    else tma_load_3d(a_dst + a_bytes, &mapB, fb, c0, n0, tap);
                    ++it;
                    if (++st == stages) {
                        st = 0;
                        ph ^= 1;
                    }
                }
            }
            s_issued = it;
        }
    } else if (warp == 5) {
        if (lane == 0) {   // MMA issuer
            const uint32_t idesc = tc_idesc(tile_n);
            int it = 0, st = 0, ph = 0, lt = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
                const int b = lt & 1;
                if (lt >= 2 && !mbar_wait_try(smem_u32(&acc_empty[b]), ((lt >> 1) - 1) & 1, TC_TIMEOUT_CYCLES)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(b * tmem_cols);
                for (int j = 0; j < niter; ++j) {
                    if (!mbar_wait_try(smem_u32(&full[st]), ph, TC_TIMEOUT_CYCLES)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(smem + st * stage_bytes), b0 = a0 + a_bytes;
                    for (int ks = 0; ks < kc / 16; ++ks)
                        tc_mma(d, tc_desc_sw(a0 + ks * 32, 2 * kc), tc_desc_sw(b0 + ks * 32, 2 * kc), idesc,
                               (j > 0 || ks > 0) ? 1u : 0u);
                    tc_commit(smem_u32(&empty[st]));
                    ++it;
                    if (++st == stages) {
                        st = 0;
                        ph ^= 1;
                    }
                }
                if (ok) tc_commit(smem_u32(&acc_full[b]));
            }
            s_consumed = it;
            tc_commit(smem_u32(done));   // arrives once every MMA issued above has completed
        }
    } else {   // epilogue: warps 0-3
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
            const int b = lt & 1;
            if (!mbar_wait_try(smem_u32(&acc_full[b]), (lt >> 1) & 1, TC_TIMEOUT_CYCLES)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m0 = (t / ntn) * TC_M, n0 = (t % ntn) * tile_n;
            const int row = m0 + warp * 32 + lane;
            tm_store_row(tmem + (uint32_t)(b * tmem_cols) + ((uint32_t)(warp * 32) << 16), row, n0,
                         min(tile_n, N - n0), tile_n, N, sbias ? s_bias + n0 : (bias ? bias + n0 : nullptr), mask, out, out_f32, relu,
                         vec_out);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(smem_u32(&acc_empty[b]));
        }
    }
    if (tid == 160) ok = mbar_wait_try(smem_u32(done), 0u, TC_TIMEOUT_CYCLES) && ok;
    ok = __syncthreads_and(ok);
    if (!ok && tid == 128) {
        // loads still in flight write this CTA's shared memory: wait for them (bounded)
        for (int it = s_consumed; it < s_issued; ++it)
            mbar_wait_try(smem_u32(&full[it % stages]), (it / stages) & 1, TC_TIMEOUT_CYCLES);
        atomicExch(&g_nop_timeout, 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * tmem_cols)
                     : "memory");
}

// Weight gradient on tcgen05: D[m = tap * cin + ci][n = co] = sum over pixels
// p of X[p + d(tap)][ci] dY[p][co], K = pixels, split over gridDim.z CTAs
// (FP32 atomics into dw).  Both operands are staged MN-major: a core matrix
// is 8 pixels (K) x 8 consecutive channels (16 bytes, M or N), exactly one
// global 16-byte vector per row; core matrices are 128 B apart along M/N
// (stride byte offset) and 128 * (rows / 8) B apart along K (leading byte
// offset).  Requires cin % 8 == 0 and cout % 8 == 0.  With db, the first
// padding row of A (row M, present when M % 128 != 0) is all ones, so row M
// of D is the bias gradient sum_p dY[p][co], added into db.
__global__ void __launch_bounds__(TC_THREADS) k_wgrad_tc(const __nv_bfloat16* __restrict__ X,
                                                         const __nv_bfloat16* __restrict__ dY, float* __restrict__ dw,
                                                         float* __restrict__ db, ConvShape s, int M, int N, int npix,
                                                         int kchunk, int tile_n, int tmem_cols) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int b_bytes = tile_n * TC_K * 2;
    unsigned char* const a_base = smem;
    unsigned char* const b_base = smem + 2 * TC_A_BYTES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * TC_A_BYTES + 2 * b_bytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * tile_n;
    const int nt = min(tile_n, N - n0), ntp = (nt + 15) & ~15;
    const int kb = blockIdx.z * kchunk, ke = min(kb + kchunk, npix);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]));
        mbar_init(smem_u32(&mbar[1]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // A rows: 16 groups of 8 channels, group g = (m0 / 8 + g): tap and channel
    const int hw = s.h * s.w;
    const int kl = tid % TC_K;                // this thread's pixel within a chunk
    const int g0 = tid / TC_K;                // its first channel group (then every TC_PIX_STEP-th)
    const uint32_t idesc = tc_idesc(ntp) | (1u << 15) | (1u << 16);     // A and B MN-major
    const int lbo_a = 128 * (TC_M / 8), lbo_b = 128 * (ntp / 8);
    const int nchunks = (ke - kb + TC_K - 1) / TC_K;
    // this thread's A vectors of chunk c (its pixel, its channel groups),
    // loaded one chunk ahead into registers
    constexpr int NA = TC_M / 8 / TC_PIX_STEP;
    uint4 va[NA];
    // the row groups' taps and channels do not change along K: decode them once
    int a_dy[NA], a_dx[NA], a_ci[NA], a_kind[NA];   // kind: 0 zero, 1 activation, 2 ones (bias row)
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        const int m = m0 + 8 * (g0 + TC_PIX_STEP * j);
        const int tap = m < M ? m / s.cin : 0;
        a_ci[j] = m - tap * s.cin;
        a_dy[j] = tap_dy(tap, s.taps);
        a_dx[j] = tap_dx(tap, s.taps);
        a_kind[j] = m < M ? 1 : (db && m == M ? 2 : 0);
    }
    // this thread's pixel of chunk c, (image, row, column), advanced by TC_K per chunk
    int c_pn = 0, c_py = 0, c_px = 0, c_at = -1;
    auto load_a = [&](int c) {
        const int p = kb + c * TC_K + kl;
        if (c_at < 0) {
            c_pn = p / hw;
            const int rem = p - c_pn * hw;
            c_py = rem / s.w;
            c_px = rem - c_py * s.w;
        } else {
            c_px += TC_K * (c - c_at);
            while (c_px >= s.w) {
                c_px -= s.w;
                if (++c_py == s.h) {
                    c_py = 0;
                    ++c_pn;
                }
            }
        }
        c_at = c;
        const bool live = p < ke;
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            va[j] = make_uint4(0u, 0u, 0u, 0u);
            if (!live) continue;
            if (a_kind[j] == 1) {
                const int yy = c_py + a_dy[j], xx = c_px + a_dx[j];
                if (yy >= 0 && yy < s.h && xx >= 0 && xx < s.w)
                    va[j] = __ldg(reinterpret_cast<const uint4*>(X + ((c_pn * s.h + yy) * s.w + xx) * s.cin + a_ci[j]));
            } else if (a_kind[j] == 2) {
                va[j] = make_uint4(0x3F80u, 0u, 0u, 0u);   // row M = ones (BF16 1.0): D[M][n] = bias gradient
            }
        }
    };
    // and its B vectors (output gradient at its pixel, channel groups g0,
    // g0 + TC_PIX_STEP, ... below ntp / 8), also one chunk ahead
    constexpr int NB = 256 / 8 / TC_PIX_STEP;
    uint4 vb[NB];
    auto load_b = [&](int c) {
        const int p = kb + c * TC_K + kl;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const int g = g0 + TC_PIX_STEP * j;
            vb[j] = make_uint4(0u, 0u, 0u, 0u);
            if (p < ke && 8 * g < nt) vb[j] = __ldg(reinterpret_cast<const uint4*>(dY + p * s.cout + n0 + 8 * g));
        }
    };
    if (nchunks > 0) {
        load_a(0);
        load_b(0);
    }
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
        const int bi = c & 1;
        if (c >= 2 && ok) ok = mbar_wait(smem_u32(&mbar[bi]), ((c - 2) >> 1) & 1);
        unsigned char* const ab = a_base + bi * TC_A_BYTES + (kl >> 3) * lbo_a + (kl & 7) * 16;
#pragma unroll
        for (int j = 0; j < NA; ++j) *reinterpret_cast<uint4*>(ab + (g0 + TC_PIX_STEP * j) * 128) = va[j];
        unsigned char* const bb = b_base + bi * b_bytes + (kl >> 3) * lbo_b + (kl & 7) * 16;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const int g = g0 + TC_PIX_STEP * j;
            if (g < ntp / 8) *reinterpret_cast<uint4*>(bb + g * 128) = vb[j];
        }
        if (c + 1 < nchunks) {
            load_a(c + 1);
            load_b(c + 1);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(a_base + bi * TC_A_BYTES), b0 = smem_u32(b_base + bi * b_bytes);
#pragma unroll
            for (int ks = 0; ks < TC_K / 16; ++ks)
                tc_mma(tmem, tc_desc(a0 + ks * 2 * lbo_a, lbo_a, 128), tc_desc(b0 + ks * 2 * lbo_b, lbo_b, 128),
                       idesc, (c > 0 || ks > 0) ? 1u : 0u);
            tc_commit(smem_u32(&mbar[bi]));
        }
    }
    if (ok && nchunks > 0) ok = mbar_wait(smem_u32(&mbar[(nchunks - 1) & 1]), ((nchunks - 1) >> 1) & 1);
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && nchunks > 0) {
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < ntp; c0 += 8) {
            uint32_t r[8];
            tc_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (c0 + j >= nt) break;
                    atomicAdd(dw + row * N + n0 + c0 + j, __uint_as_float(r[j]));
                }
            } else if (db && row == M) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (c0 + j >= nt) break;
                    atomicAdd(db + n0 + c0 + j, __uint_as_float(r[j]));
                }
            }
        }
    } else if (!ok && tid == 0) {
        atomicExch(&g_nop_timeout, 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// ---------------------------------------------------------------- TMA weight gradient
// Weight gradient fed by the Tensor Memory Accelerator: D[m][n] = sum over
// pixels p of A[m][p] B[n][p] with both operands MN-major (channels
// contiguous, pixels along K), read straight from the NHWC tensors.  The M
// rows of a tile are "atoms" of AW channels (AW = 32 with the 64-byte
// swizzle, or 64 with the 128-byte one): atom a = (tap a / apt, channels
// (a % apt) AW ...), loaded per 64-pixel K chunk as one 4-D box of X shifted
// by the tap (zero fill at the image borders and past the last channel).
// B atoms are BW-channel boxes of dY.  The canonical MN-major swizzled
// layout: an atom's 64 K rows of 2 AW bytes in 8-row groups (stride byte
// offset 16 AW), atoms one box apart (leading byte offset).  Slots past the
// last atom hold zeros; with db the first of them is a row of ones, whose D
// row is the bias gradient sum_p dY[p][n].  Those slots are written once per
// stage before the loop and never loaded.  Roles and bounded waits as in
// k_conv_tma's first form: thread 0 issues the copies into a ring of
// `stages` buffers, thread 32 the four K = 16 MMAs per chunk; the four warps
// add their rows to dw (FP32 atomics: the pixel sum is split over gridDim.z).
constexpr int WG_K = 64;   // pixels per K chunk

__device__ __forceinline__ uint64_t tc_desc_mn(uint32_t addr, uint32_t lbo, int row_bytes) {
    const uint64_t mode = row_bytes == 128 ? 2ull : 4ull;
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((8 * row_bytes) >> 4) << 32) | (1ull << 46) | (mode << 61);
}

__global__ void __launch_bounds__(TC_THREADS) k_wgrad_tma(const __grid_constant__ CUtensorMap mapA,
                                                          const __grid_constant__ CUtensorMap mapB,
                                                          float* __restrict__ dw, float* __restrict__ db, ConvShape s,
                                                          int aw, int apt, int bw, int tile_n, int tmem_cols,
                                                          int stages, int chunks_per_cta, int nchunks, int ones_atom) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* const smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int a_atoms = TC_M / aw, atom_b = WG_K * aw * 2, a_bytes = a_atoms * atom_b;
    const int b_atoms = tile_n / bw, batom_b = WG_K * bw * 2;
    const int stage_bytes = a_bytes + b_atoms * batom_b;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + stages * stage_bytes);
    uint64_t* empty = full + stages;
    uint64_t* done = empty + stages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int s_issued, s_consumed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int atom0 = blockIdx.x * a_atoms, n0 = blockIdx.y * tile_n;
    const int atoms = s.taps * apt;
    const int na_real = max(0, min(a_atoms, atoms - atom0));
    const int c_begin = blockIdx.z * chunks_per_cta, c_end = min(nchunks, c_begin + chunks_per_cta);
    const int hw = s.h * s.w;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < stages; ++i) {
            mbar_init(smem_u32(&full[i]));
            mbar_init(smem_u32(&empty[i]));
        }
        mbar_init(smem_u32(done));
        s_issued = 0;
        s_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // slots past the last atom: zeros, and the row of ones (element (k, 0) of
    // the atom for every K row k, at its swizzled place: the 16-byte chunk
    // index of row k is XORed with k / 2 mod 4 (64-byte rows) or k mod 8 (128-byte))
    for (int st = 0; st < stages; ++st)
        for (int j = na_real; j < a_atoms; ++j) {
            unsigned char* at = smem + st * stage_bytes + j * atom_b;
            for (int i = tid; i < atom_b / 16; i += TC_THREADS) reinterpret_cast<uint4*>(at)[i] = make_uint4(0u, 0u, 0u, 0u);
        }
    __syncthreads();
    if (ones_atom >= atom0 + na_real && ones_atom < atom0 + a_atoms && tid < WG_K)
        for (int st = 0; st < stages; ++st) {
            const int k = tid, rb = 2 * aw;
            const int chunk = rb == 128 ? (k & 7) : ((k >> 1) & 3);
            unsigned char* at = smem + st * stage_bytes + (ones_atom - atom0) * atom_b;
            *reinterpret_cast<__nv_bfloat16*>(at + k * rb + 16 * chunk) = __float2bfloat16(1.0f);
        }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    bool ok = true;
    const int niter = c_end - c_begin;
    if (tid == 0) {   // producer
        int it = 0;
        for (; it < niter; ++it) {
            const int st = it % stages;
            if (it >= stages && !mbar_wait_try(smem_u32(&empty[st]), ((it / stages) - 1) & 1, TC_TIMEOUT_CYCLES)) {
                ok = false;
                break;
            }
            const int p0 = (c_begin + it) * WG_K, img = p0 / hw, rem = p0 - img * hw;
            const int h0 = rem / s.w, w0 = rem - h0 * s.w;
            const uint32_t fb = smem_u32(&full[st]), base = smem_u32(smem + st * stage_bytes);
            mbar_expect_tx(fb, (uint32_t)(na_real * atom_b + b_atoms * batom_b));
            for (int j = 0; j < na_real; ++j) {
                const int a = atom0 + j, tap = a / apt, c0 = (a - tap * apt) * aw;
                tma_load_4d(base + j * atom_b, &mapA, fb, c0, w0 + tap_dx(tap, s.taps), h0 + tap_dy(tap, s.taps), img);
            }
            for (int j = 0; j < b_atoms; ++j) tma_load_4d(base + a_bytes + j * batom_b, &mapB, fb, n0 + j * bw, w0, h0, img);
        }
        s_issued = it;
    } else if (tid == 32) {   // MMA issuer
        const uint32_t idesc = tc_idesc(tile_n) | (1u << 15) | (1u << 16);   // A and B MN-major
        int it = 0;
        for (; it < niter; ++it) {
            const int st = it % stages;
            if (!mbar_wait_try(smem_u32(&full[st]), (it / stages) & 1, TC_TIMEOUT_CYCLES)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(smem + st * stage_bytes), b0 = a0 + a_bytes;
#pragma unroll
            for (int ks = 0; ks < WG_K / 16; ++ks)   // 16 K rows = two 8-row groups
                tc_mma(tmem, tc_desc_mn(a0 + ks * 32 * aw, atom_b, 2 * aw), tc_desc_mn(b0 + ks * 32 * bw, batom_b, 2 * bw),
                       idesc, (it > 0 || ks > 0) ? 1u : 0u);
            tc_commit(smem_u32(&empty[st]));
        }
        s_consumed = it;
        tc_commit(smem_u32(done));
    }
    ok = ok && mbar_wait_try(smem_u32(done), 0u, TC_TIMEOUT_CYCLES);
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0) {
        for (int it = s_consumed; it < s_issued; ++it)
            mbar_wait_try(smem_u32(&full[it % stages]), (it / stages) & 1, TC_TIMEOUT_CYCLES);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && niter > 0) {
        const int r = warp * 32 + lane, atom = atom0 + r / aw, within = r - (r / aw) * aw;
        float* dst = nullptr;
        if (atom < atoms) {
            const int tap = atom / apt, ci = (atom - tap * apt) * aw + within;
            if (ci < s.cin) dst = dw + (size_t)(tap * s.cin + ci) * s.cout + n0;
        } else if (db && atom == ones_atom && within == 0) {
            dst = db + n0;
        }
        const int nt = min(tile_n, s.cout - n0);
        for (int c0 = 0; c0 < tile_n; c0 += 32) {
            uint32_t v[32];
            tc_ld32_nowait(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            tc_wait_ld();
            if (dst)
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c0 + j < nt) atomicAdd(dst + c0 + j, __uint_as_float(v[j]));
        }
    } else if (!ok && tid == 0) {
        atomicExch(&g_nop_timeout, 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// Streaming multiprocessors of the current device (looked up once).
int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) ==
                                                      cudaSuccess && v > 0)
            n = v;
        else
            n = 148;
    }
    return n;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependency on libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// BF16 tensor map with the given swizzle and zero fill outside the tensor;
// dims[0] is the contiguous dimension, strides[i] the byte stride of dims[i + 1].
bool encode_map(CUtensorMap* map, const void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                const cuuint32_t* box, CUtensorMapSwizzle swizzle) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box,
               ones, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launches the TMA-fed tcgen05 kernel; false when the shape is not one it
// takes: tiles must be whole rows (width a multiple of 128, or a divisor of
// 128 with the height a multiple of 128 / width), channel counts multiples
// of 8 (16-byte strides), operands 16-byte aligned.
template <int MODE>
bool launch_tma(const void* A, const void* B, const float* bias, const void* mask, void* out, int out_f32, int relu,
                ConvShape s, long long M, long long N, cudaStream_t st, int* rc) {
    const int C = MODE == FWD ? s.cin : s.cout;
    if (C % 8 || N % 8 || !aligned16(A) || !aligned16(B) || M <= 0 || N <= 0) return false;
    if (s.taps != 9 && s.taps != 1) return false;
    int wbox, hbox;
    if (s.w >= TC_M) {
        if (s.w % TC_M) return false;
        wbox = TC_M;
        hbox = 1;
    } else {
        if (TC_M % s.w || s.h % (TC_M / s.w)) return false;
        wbox = s.w;
        hbox = TC_M / s.w;
    }
    const long long npix = (long long)s.n * s.h * s.w;
    const long long cmax = s.cin > s.cout ? s.cin : s.cout;
    if (npix * cmax * s.taps >= 2147483647LL || M * N >= 2147483647LL) return false;
    const int tile_n = N <= 256 ? (int)((N + 15) & ~15LL) : 256;
    int cols = 32;
    while (cols < tile_n) cols <<= 1;
    // 32-channel chunks (64-byte rows) up to 32 channels, else 64-channel
    // ones (128-byte rows).  For channel counts that are odd multiples of 32
    // the last 64-wide box runs past the last channel (filled by the hardware);
    // 32-wide chunks there measured slower over the training step (1.30 ms
    // against 1.27) because of the extra MMA groups and stages.  Keeping the
    // weights of a one-N-tile layer resident in shared memory instead of
    // streaming them with each stage measured the same (L2 serves them).
    const int kc = C <= 32 ? 32 : 64;
    const int cchunks = (C + kc - 1) / kc;
    // two CTAs per SM (two accumulator buffers each) while both fit in TMEM
    const int per_sm = 2 * cols <= 256 ? 2 : 1;
    const size_t stage_bytes = (size_t)TC_M * kc * 2 + (size_t)tile_n * kc * 2;
    // dynamic shared memory per CTA: what is left of the SM's 228 KB after the
    // static bias stage (TM_BIAS_MAX floats) and the per-CTA reservation
    const size_t budget = (per_sm == 2 ? 104 : 214) * 1024 - 1024 - 128;
    const int stages = (int)std::min<size_t>(CLB_TM_MAX_STAGES, budget / stage_bytes);
    if (stages < 2) return false;
    CUtensorMap ma, mb;
    const CUtensorMapSwizzle sw = kc == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    {
        const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)s.w, (cuuint64_t)s.h, (cuuint64_t)s.n};
        const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)s.w * C * 2, (cuuint64_t)s.h * s.w * C * 2};
        const cuuint32_t box[4] = {(cuuint32_t)kc, (cuuint32_t)wbox, (cuuint32_t)hbox, 1};
        if (!encode_map(&ma, A, 4, dims, strides, box, sw)) return false;
    }
    if (MODE == FWD) {   // W^T [cout][taps * cin] as (cin, taps, cout)
        const cuuint64_t dims[3] = {(cuuint64_t)s.cin, (cuuint64_t)s.taps, (cuuint64_t)s.cout};
        const cuuint64_t strides[2] = {(cuuint64_t)s.cin * 2, (cuuint64_t)s.taps * s.cin * 2};
        const cuuint32_t box[3] = {(cuuint32_t)kc, 1, (cuuint32_t)tile_n};
        if (!encode_map(&mb, B, 3, dims, strides, box, sw)) return false;
    } else {             // W [taps * cin][cout] as (cout, cin, taps)
        const cuuint64_t dims[3] = {(cuuint64_t)s.cout, (cuuint64_t)s.cin, (cuuint64_t)s.taps};
        const cuuint64_t strides[2] = {(cuuint64_t)s.cout * 2, (cuuint64_t)s.cin * s.cout * 2};
        const cuuint32_t box[3] = {(cuuint32_t)kc, (cuuint32_t)tile_n, 1};
        if (!encode_map(&mb, B, 3, dims, strides, box, sw)) return false;
    }
    const size_t smem = 1024 + stages * stage_bytes + (2 * stages + 5) * 8 + 16;
    if (cudaFuncSetAttribute(k_conv_tma<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        *rc = CLB_NOP_ERR_CUDA;
        return true;
    }
    const int ntn = (int)((N + tile_n - 1) / tile_n);
    const long long ntiles = (M / TC_M) * ntn;
    const unsigned grid = (unsigned)std::min<long long>(ntiles, (long long)sm_count() * per_sm);
    const int vec_out = N % 8 == 0 && aligned16(out) && (!mask || aligned16(mask));
    k_conv_tma<MODE><<<grid, TM_THREADS, smem, st>>>(ma, mb, bias, (const __nv_bfloat16*)mask, out, out_f32, relu, s,
                                                      (int)M, (int)N, tile_n, cols, vec_out, stages, cchunks, kc,
                                                      (int)ntiles, ntn);
    *rc = cudaGetLastError() == cudaSuccess ? CLB_NOP_OK : CLB_NOP_ERR_CUDA;
    return true;
}

// Launches the tcgen05 kernel; false when the shape is not one it takes.
template <int MODE>
bool launch_tc(const void* A, const void* B, const float* bias, const void* mask, void* out, int out_f32, int relu,
               ConvShape s, long long M, long long N, long long K, cudaStream_t st, int* rc) {
    const int C = MODE == FWD ? s.cin : s.cout;
    if (C % 8 || !aligned16(A) || !aligned16(B) || M <= 0 || N <= 0 || K <= 0) return false;
    const long long npix = (long long)s.n * s.h * s.w;
    const long long cmax = s.cin > s.cout ? s.cin : s.cout;
    if (npix * cmax * s.taps >= 2147483647LL || M * N >= 2147483647LL) return false;
    const int tile_n = N <= 256 ? (int)((N + 15) & ~15LL) : 256;
    int cols = 32;
    while (cols < tile_n) cols <<= 1;
    const size_t smem = 2 * (size_t)TC_A_BYTES + 2 * (size_t)tile_n * TC_K * 2 + 32;
    if (cudaFuncSetAttribute(k_conv_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * TC_A_BYTES + 2 * 256 * TC_K * 2 + 32) != cudaSuccess) {
        *rc = CLB_NOP_ERR_CUDA;
        return true;
    }
    const dim3 grid((unsigned)((M + TC_M - 1) / TC_M), (unsigned)((N + tile_n - 1) / tile_n));
    // 16-byte epilogue stores: rows of N outputs stay 16-byte aligned when N % 8 == 0
    const int vec_out = N % 8 == 0 && aligned16(out) && (!mask || aligned16(mask));
    k_conv_tc<MODE><<<grid, TC_THREADS, smem, st>>>((const __nv_bfloat16*)A, (const __nv_bfloat16*)B, bias,
                                                    (const __nv_bfloat16*)mask, out, out_f32, relu, s, (int)M, (int)N,
                                                    (int)K, tile_n, cols, vec_out);
    *rc = cudaGetLastError() == cudaSuccess ? CLB_NOP_OK : CLB_NOP_ERR_CUDA;
    return true;
}

// Launches the TMA-fed weight gradient; false when the shape is not one it
// takes (chunks of 64 pixels inside one image: width a multiple of 64, or a
// divisor of 64 with the height a multiple of 64 / width; channel counts
// multiples of 8, at most 256 outputs per tile).  *bias_done tells whether
// db was filled through the row of ones (no free atom slot: not).
bool launch_wgrad_tma(const void* x, const void* dy, float* dw, float* db, ConvShape s, int splitk, cudaStream_t st,
                      int* rc, bool* bias_done) {
    *bias_done = false;
    if (s.cin % 8 || s.cout % 8 || !aligned16(x) || !aligned16(dy)) return false;
    if (s.taps != 9 && s.taps != 1) return false;
    int wbox, hbox;
    if (s.w >= WG_K) {
        if (s.w % WG_K) return false;
        wbox = WG_K;
        hbox = 1;
    } else {
        if (WG_K % s.w || s.h % (WG_K / s.w)) return false;
        wbox = s.w;
        hbox = WG_K / s.w;
    }
    const long long npix = (long long)s.n * s.h * s.w;
    if (npix * (s.cin > s.cout ? s.cin : s.cout) * s.taps >= 2147483647LL) return false;
    // 32-channel atoms unless 64-channel ones waste no more rows (fewer boxes)
    const int aw = (s.cin + 31) / 32 * 32 < (s.cin + 63) / 64 * 64 ? 32 : 64;
    const int apt = (s.cin + aw - 1) / aw, atoms = s.taps * apt;
    const int a_atoms = TC_M / aw;
    const int bw = s.cout <= 32 ? 32 : 64, batoms_all = (s.cout + bw - 1) / bw;   // as the convolution's chunks
    const int b_atoms = std::min(batoms_all, 256 / bw), tile_n = b_atoms * bw;
    const int ntn = (batoms_all + b_atoms - 1) / b_atoms;
    const int ones_atom = (db && atoms % a_atoms) ? atoms : -1;
    const int mtiles = (atoms + a_atoms - 1) / a_atoms;
    int cols = 32;
    while (cols < tile_n) cols <<= 1;
    const size_t stage_bytes = (size_t)TC_M * 2 * WG_K + (size_t)tile_n * 2 * WG_K;
    const int stages = (int)std::min<size_t>(CLB_WG_MAX_STAGES, std::max<size_t>(2, (100 * 1024) / stage_bytes));
    const size_t smem = 1024 + stages * stage_bytes + (2 * stages + 1) * 8 + 16;
    const int nchunks = (int)(npix / WG_K);
    const long long tiles = (long long)mtiles * ntn;
    if (splitk < 1) {
        // automatic: one wave of two CTAs per SM (the shared-memory limit), each
        // with at least 4 chunks
        const long long want = std::max(1LL, 2LL * sm_count() / tiles);
        splitk = (int)std::max(1LL, std::min(want, (long long)nchunks / 4));
    }
    const int per = (nchunks + splitk - 1) / splitk, gz = (nchunks + per - 1) / per;
    if (gz > 65535 || mtiles > 65535) return false;
    CUtensorMap ma, mb;
    {
        const cuuint64_t dims[4] = {(cuuint64_t)s.cin, (cuuint64_t)s.w, (cuuint64_t)s.h, (cuuint64_t)s.n};
        const cuuint64_t strides[3] = {(cuuint64_t)s.cin * 2, (cuuint64_t)s.w * s.cin * 2,
                                       (cuuint64_t)s.h * s.w * s.cin * 2};
        const cuuint32_t box[4] = {(cuuint32_t)aw, (cuuint32_t)wbox, (cuuint32_t)hbox, 1};
        if (!encode_map(&ma, x, 4, dims, strides, box, aw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B))
            return false;
    }
    {
        const cuuint64_t dims[4] = {(cuuint64_t)s.cout, (cuuint64_t)s.w, (cuuint64_t)s.h, (cuuint64_t)s.n};
        const cuuint64_t strides[3] = {(cuuint64_t)s.cout * 2, (cuuint64_t)s.w * s.cout * 2,
                                       (cuuint64_t)s.h * s.w * s.cout * 2};
        const cuuint32_t box[4] = {(cuuint32_t)bw, (cuuint32_t)wbox, (cuuint32_t)hbox, 1};
        if (!encode_map(&mb, dy, 4, dims, strides, box, bw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B))
            return false;
    }
    if (cudaFuncSetAttribute(k_wgrad_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        *rc = CLB_NOP_ERR_CUDA;
        return true;
    }
    const dim3 grid((unsigned)mtiles, (unsigned)ntn, (unsigned)gz);
    k_wgrad_tma<<<grid, TC_THREADS, smem, st>>>(ma, mb, dw, db, s, aw, apt, bw, tile_n, cols, stages, per, nchunks,
                                                ones_atom);
    *rc = cudaGetLastError() == cudaSuccess ? CLB_NOP_OK : CLB_NOP_ERR_CUDA;
    *bias_done = ones_atom >= 0;
    return true;
}

// Launches the tcgen05 weight gradient; false when the shape is not one it takes.
bool launch_wgrad_tc(const void* x, const void* dy, float* dw, float* db, ConvShape s, int splitk, cudaStream_t st,
                     int* rc) {
    if (s.cin % 8 || s.cout % 8 || !aligned16(x) || !aligned16(dy)) return false;
    const long long npix = (long long)s.n * s.h * s.w;
    const long long cmax = s.cin > s.cout ? s.cin : s.cout;
    const long long M = (long long)s.taps * s.cin, N = s.cout;
    if (db && M % TC_M == 0) return false;   // no free row for the bias
    if (npix * cmax * s.taps >= 2147483647LL || M * N >= 2147483647LL) return false;
    const int tile_n = N <= 256 ? (int)((N + 15) & ~15LL) : 256;
    int cols = 32;
    while (cols < tile_n) cols <<= 1;
    const long long tiles = ((M + TC_M - 1) / TC_M) * ((N + tile_n - 1) / tile_n);
    if (splitk < 1) {
        // automatic: about four CTAs per SM, each with at least 8 K chunks
        const long long want = (4LL * 152 + tiles - 1) / tiles, most = (npix + 8 * TC_K - 1) / (8 * TC_K);
        splitk = (int)std::max(1LL, std::min(want, most));
    }
    long long kchunk = (npix + splitk - 1) / splitk;
    kchunk = (kchunk + TC_K - 1) / TC_K * TC_K;
    const long long gz = (npix + kchunk - 1) / kchunk;
    if (gz > 65535) return false;
    const size_t smem = 2 * (size_t)TC_A_BYTES + 2 * (size_t)tile_n * TC_K * 2 + 32;
    if (cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * TC_A_BYTES + 2 * 256 * TC_K * 2 + 32) != cudaSuccess) {
        *rc = CLB_NOP_ERR_CUDA;
        return true;
    }
    const dim3 grid((unsigned)((M + TC_M - 1) / TC_M), (unsigned)((N + tile_n - 1) / tile_n), (unsigned)gz);
    k_wgrad_tc<<<grid, TC_THREADS, smem, st>>>((const __nv_bfloat16*)x, (const __nv_bfloat16*)dy, dw, db, s, (int)M,
                                               (int)N, (int)npix, (int)kchunk, tile_n, cols);
    *rc = cudaGetLastError() == cudaSuccess ? CLB_NOP_OK : CLB_NOP_ERR_CUDA;
    return true;
}

// ---------------------------------------------------------------- elementwise
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dy, float* __restrict__ db, long long npix, int c) {
    // one block per 256 pixels x all channels: per-channel partial sums, atomics
    const long long p0 = (long long)blockIdx.x * 256;
    for (int ch = threadIdx.x; ch < c; ch += blockDim.x) {
        float s = 0.0f;
        const long long p1 = p0 + 256 < npix ? p0 + 256 : npix;
        for (long long p = p0; p < p1; ++p) s += __bfloat162float(dy[p * c + ch]);
        atomicAdd(db + ch, s);
    }
}

__global__ void k_pool2_fwd(const __nv_bfloat16* __restrict__ x, __nv_bfloat16* __restrict__ y, int n, int h, int w, int c) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ho = h / 2, wo = w / 2;
    if (i >= (long long)n * ho * wo * c) return;
    const int ch = (int)(i % c);
    long long p = i / c;
    const int xo = (int)(p % wo);
    p /= wo;
    const int yo = (int)(p % ho);
    const int b = (int)(p / ho);
    const long long base = (((long long)b * h + 2 * yo) * w + 2 * xo) * c + ch;
    const float s = __bfloat162float(x[base]) + __bfloat162float(x[base + c]) + __bfloat162float(x[base + (long long)w * c]) +
                    __bfloat162float(x[base + (long long)w * c + c]);
    y[i] = __float2bfloat16(0.25f * s);
}

__global__ void k_pool2_bwd(const __nv_bfloat16* __restrict__ dy, __nv_bfloat16* __restrict__ dx, int n, int h, int w, int c) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * h * w * c) return;
    const int ch = (int)(i % c);
    long long p = i / c;
    const int x = (int)(p % w);
    p /= w;
    const int y = (int)(p % h);
    const int b = (int)(p / h);
    const int ho = h / 2, wo = w / 2;
    dx[i] = __float2bfloat16(0.25f * __bfloat162float(dy[(((long long)b * ho + y / 2) * wo + x / 2) * c + ch]));
}

__global__ void k_up2_fwd(const __nv_bfloat16* __restrict__ x, __nv_bfloat16* __restrict__ y, int n, int h, int w, int c) {
    // x: (n, h, w, c) -> y: (n, 2h, 2w, c), nearest
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int H = 2 * h, W = 2 * w;
    if (i >= (long long)n * H * W * c) return;
    const int ch = (int)(i % c);
    long long p = i / c;
    const int X = (int)(p % W);
    p /= W;
    const int Y = (int)(p % H);
    const int b = (int)(p / H);
    y[i] = x[(((long long)b * h + Y / 2) * w + X / 2) * c + ch];
}

__global__ void k_up2_bwd(const __nv_bfloat16* __restrict__ dy, __nv_bfloat16* __restrict__ dx, int n, int h, int w, int c) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * h * w * c) return;
    const int ch = (int)(i % c);
    long long p = i / c;
    const int x = (int)(p % w);
    p /= w;
    const int y = (int)(p % h);
    const int b = (int)(p / h);
    const int W = 2 * w;
    const long long base = (((long long)b * 2 * h + 2 * y) * W + 2 * x) * c + ch;
    const float s = __bfloat162float(dy[base]) + __bfloat162float(dy[base + c]) + __bfloat162float(dy[base + (long long)W * c]) +
                    __bfloat162float(dy[base + (long long)W * c + c]);
    dx[i] = __float2bfloat16(s);
}

// Channel concatenation of a (npix, ca) and b (npix, cb) into y (npix, ca + cb), and its inverse.
__global__ void k_concat(const __nv_bfloat16* __restrict__ a, const __nv_bfloat16* __restrict__ b, __nv_bfloat16* __restrict__ y,
                         long long npix, int ca, int cb, int inverse) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = ca + cb;
    if (i >= npix * c) return;
    const long long p = i / c;
    const int ch = (int)(i - p * c);
    if (!inverse) y[i] = ch < ca ? a[p * ca + ch] : b[p * cb + ch - ca];
    else if (ch < ca) const_cast<__nv_bfloat16*>(a)[p * ca + ch] = y[i];
    else const_cast<__nv_bfloat16*>(b)[p * cb + ch - ca] = y[i];
}

// Channel-weighted mean squared error over n values (nch channels, fastest
// index): loss += sum_i w[c] (pred_i - target_i)^2 / n, grad_i = 2 w[c]
// (pred_i - target_i) / n as BF16; w = NULL means all weights 1.
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ target, const float* __restrict__ wch,
                      int nch, __nv_bfloat16* __restrict__ grad, float* __restrict__ loss, long long n) {
    __shared__ float sh[32];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.0f;
    if (i < n) {
        const float wc = wch ? wch[i % nch] : 1.0f;
        const float d = pred[i] - target[i];
        grad[i] = __float2bfloat16(2.0f * wc * d / (float)n);
        e = wc * d * d / (float)n;
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x < 32) {
        e = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
        if (threadIdx.x == 0) atomicAdd(loss, e);
    }
}

// Adam on FP32 master weights; refreshes the BF16 working copy.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       __nv_bfloat16* __restrict__ wb, long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16(wi);
}

__global__ void k_cast_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16(x[i]);
}

unsigned nblk(long long n) { return (unsigned)((n + 255) / 256); }

// ------------------------------------------------ 16-byte (8-channel) forms
// The same operations, one uint4 of eight BF16 channels per thread, taken
// when every channel count is a multiple of 8 and every pointer is 16-byte
// aligned (all layers of the network); the scalar kernels above stay for the
// other shapes.
__device__ __forceinline__ void unpack8(const uint4 v, float (&f)[8]) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 t = __bfloat1622float2(h[j]);
        f[2 * j] = t.x;
        f[2 * j + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
    uint4 v;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
    return v;
}

// n * h * w pixels of G = c / 8 vectors; vector index i -> (pixel, group)
__global__ void k_pool2_fwd8(const uint4* __restrict__ x, uint4* __restrict__ y, int n, int h, int w, int G) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ho = h / 2, wo = w / 2;
    if (i >= (long long)n * ho * wo * G) return;
    const int g = (int)(i % G);
    long long p = i / G;
    const int xo = (int)(p % wo);
    p /= wo;
    const int yo = (int)(p % ho);
    const int b = (int)(p / ho);
    const long long base = (((long long)b * h + 2 * yo) * w + 2 * xo) * G + g;
    float a[8], t[8];
    unpack8(x[base], a);
    unpack8(x[base + G], t);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] += t[j];
    unpack8(x[base + (long long)w * G], t);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] += t[j];
    unpack8(x[base + (long long)w * G + G], t);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 0.25f * (a[j] + t[j]);
    y[i] = pack8(a);
}

__global__ void k_pool2_bwd8(const uint4* __restrict__ dy, uint4* __restrict__ dx, int n, int h, int w, int G) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * h * w * G) return;
    const int g = (int)(i % G);
    long long p = i / G;
    const int x = (int)(p % w);
    p /= w;
    const int y = (int)(p % h);
    const int b = (int)(p / h);
    float a[8];
    unpack8(dy[(((long long)b * (h / 2) + y / 2) * (w / 2) + x / 2) * G + g], a);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] *= 0.25f;
    dx[i] = pack8(a);
}

__global__ void k_up2_fwd8(const uint4* __restrict__ x, uint4* __restrict__ y, int n, int h, int w, int G) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int H = 2 * h, W = 2 * w;
    if (i >= (long long)n * H * W * G) return;
    const int g = (int)(i % G);
    long long p = i / G;
    const int X = (int)(p % W);
    p /= W;
    const int Y = (int)(p % H);
    const int b = (int)(p / H);
    y[i] = x[(((long long)b * h + Y / 2) * w + X / 2) * G + g];
}

__global__ void k_up2_bwd8(const uint4* __restrict__ dy, uint4* __restrict__ dx, int n, int h, int w, int G) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * h * w * G) return;
    const int g = (int)(i % G);
    long long p = i / G;
    const int x = (int)(p % w);
    p /= w;
    const int y = (int)(p % h);
    const int b = (int)(p / h);
    const int W = 2 * w;
    const long long base = (((long long)b * 2 * h + 2 * y) * W + 2 * x) * G + g;
    float a[8], t[8];
    unpack8(dy[base], a);
    unpack8(dy[base + G], t);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] += t[j];
    unpack8(dy[base + (long long)W * G], t);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] += t[j];
    unpack8(dy[base + (long long)W * G + G], t);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] += t[j];
    dx[i] = pack8(a);
}

// ga = ca / 8 and gb = cb / 8 vectors per pixel
__global__ void k_concat8(uint4* __restrict__ a, uint4* __restrict__ b, uint4* __restrict__ y, long long npix, int ga,
                          int gb, int inverse) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int G = ga + gb;
    if (i >= npix * G) return;
    const long long p = i / G;
    const int g = (int)(i - p * G);
    uint4* src = g < ga ? a + p * ga + g : b + p * gb + (g - ga);
    if (!inverse) y[i] = *src;
    else *src = y[i];
}

__global__ void k_add_mask8(const uint4* __restrict__ d1, const uint4* __restrict__ d2, const uint4* __restrict__ a,
                            uint4* __restrict__ out, long long n8) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n8) return;
    float v[8], t[8];
    unpack8(d1[i], v);
    if (d2) {
        unpack8(d2[i], t);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] += t[j];
    }
    if (a) {
        unpack8(a[i], t);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (!(t[j] > 0.0f)) v[j] = 0.0f;
    }
    out[i] = pack8(v);
}

// Bias gradient db[ch] += sum_p dy[p][ch] for c % 8 == 0: a grid-stride loop
// over 16-byte vectors with a stride that is a multiple of G = c / 8, so every
// thread keeps one channel group; per-block sums of the threads of each group
// (shared memory), then one FP32 atomic per block and channel.
constexpr int BG_THREADS = 256;
constexpr int BG_BLOCKS = 2 * 152;

__global__ void __launch_bounds__(BG_THREADS) k_bias_grad8(const uint4* __restrict__ dy, float* __restrict__ db,
                                                            long long n8, int G) {
    __shared__ float part[BG_THREADS][9];
    const int T = (BG_THREADS / G) * G;              // threads in use: a multiple of G
    const int t = threadIdx.x;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (t < T) {
        const long long stride = (long long)T * gridDim.x;
        for (long long i = (long long)blockIdx.x * T + t; i < n8; i += stride) {
            float v[8];
            unpack8(dy[i], v);
#pragma unroll
            for (int j = 0; j < 8; ++j) s[j] += v[j];
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) part[t][j] = s[j];
    __syncthreads();
    // thread (g, j) of the first 8 G sums lane j of group g over the block's threads t = g (mod G)
    for (int q = t; q < 8 * G; q += BG_THREADS) {
        const int g = q >> 3, j = q & 7;
        float acc = 0.0f;
        for (int u = g; u < T; u += G) acc += part[u][j];
        atomicAdd(db + 8 * g + j, acc);
    }
}

// Weight gradient of a 1x1 convolution with few outputs (the network's head):
// dw[ci][co] += sum_p x[p][ci] dy[p][co] for CIN inputs (a multiple of 8) and
// COUT outputs, and (db not NULL) db[co] += sum_p dy[p][co]; each thread
// accumulates all products over a strided set of pixels, then warp shuffles
// and one atomic per block and value.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_wgrad_small(const __nv_bfloat16* __restrict__ x,
                                                     const __nv_bfloat16* __restrict__ dy, float* __restrict__ dw,
                                                     float* __restrict__ db, long long npix) {
    constexpr int NA = CIN * COUT + COUT;       // weights, then the bias (sum of dy)
    __shared__ float red[8][NA];
    float acc[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) acc[k] = 0.0f;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (long long)blockDim.x * gridDim.x) {
        float d[COUT];
#pragma unroll
        for (int o = 0; o < COUT; ++o) {
            d[o] = __bfloat162float(dy[p * COUT + o]);
            acc[CIN * COUT + o] += d[o];
        }
        const uint4* xr = reinterpret_cast<const uint4*>(x + p * CIN);
#pragma unroll
        for (int v = 0; v < CIN / 8; ++v) {
            float xv[8];
            unpack8(xr[v], xv);
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int o = 0; o < COUT; ++o) acc[(8 * v + j) * COUT + o] = fmaf(xv[j], d[o], acc[(8 * v + j) * COUT + o]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NA; ++k) {
        float v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NA; k += blockDim.x) {
        float v = 0.0f;
        for (int wi = 0; wi < 8; ++wi) v += red[wi][k];
        if (k < CIN * COUT) atomicAdd(dw + k, v);
        else if (db) atomicAdd(db + (k - CIN * COUT), v);
    }
}

// Input gradient of a 1x1 convolution with few outputs (the network's head):
// dx[p][ci] = sum_co dy[p][co] w[ci][co], zeroed where mask[p][ci] <= 0 (mask
// may be NULL); one pixel per thread, the CIN x COUT weights in shared memory.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_dgrad_small(const __nv_bfloat16* __restrict__ dy,
                                                     const __nv_bfloat16* __restrict__ w,
                                                     const __nv_bfloat16* __restrict__ mask,
                                                     __nv_bfloat16* __restrict__ dx, long long npix) {
    __shared__ float sw[CIN * COUT];
    for (int k = threadIdx.x; k < CIN * COUT; k += blockDim.x) sw[k] = __bfloat162float(w[k]);
    __syncthreads();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    float d[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) d[o] = __bfloat162float(dy[p * COUT + o]);
#pragma unroll
    for (int v = 0; v < CIN / 8; ++v) {
        float r[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float a = 0.0f;
#pragma unroll
            for (int o = 0; o < COUT; ++o) a = fmaf(d[o], sw[(8 * v + j) * COUT + o], a);
            r[j] = a;
        }
        if (mask) {
            float m[8];
            unpack8(reinterpret_cast<const uint4*>(mask + p * CIN)[v], m);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (!(m[j] > 0.0f)) r[j] = 0.0f;
        }
        reinterpret_cast<uint4*>(dx + p * CIN)[v] = pack8(r);
    }
}

// Launches k_dgrad_small for the shapes it is instantiated for; false otherwise.
bool launch_dgrad_small(const void* dy, const void* w, const void* mask, void* dx, ConvShape s, cudaStream_t st,
                        int* rc) {
    if (s.taps != 1 || !aligned16(dx) || (mask && !aligned16(mask))) return false;
    const long long npix = (long long)s.n * s.h * s.w;
    const unsigned grid = (unsigned)((npix + 255) / 256);
    const __nv_bfloat16 *dyb = (const __nv_bfloat16*)dy, *wb = (const __nv_bfloat16*)w,
                        *mb = (const __nv_bfloat16*)mask;
    __nv_bfloat16* dxb = (__nv_bfloat16*)dx;
    if (s.cout == 4 && s.cin == 8) k_dgrad_small<8, 4><<<grid, 256, 0, st>>>(dyb, wb, mb, dxb, npix);
    else if (s.cout == 4 && s.cin == 16) k_dgrad_small<16, 4><<<grid, 256, 0, st>>>(dyb, wb, mb, dxb, npix);
    else if (s.cout == 4 && s.cin == 24) k_dgrad_small<24, 4><<<grid, 256, 0, st>>>(dyb, wb, mb, dxb, npix);
    else if (s.cout == 4 && s.cin == 32) k_dgrad_small<32, 4><<<grid, 256, 0, st>>>(dyb, wb, mb, dxb, npix);
    else return false;
    *rc = cudaGetLastError() == cudaSuccess ? CLB_NOP_OK : CLB_NOP_ERR_CUDA;
    return true;
}

// Launches k_wgrad_small for the shapes it is instantiated for; false otherwise.
bool launch_wgrad_small(const void* x, const void* dy, float* dw, float* db, ConvShape s, cudaStream_t st, int* rc) {
    if (s.taps != 1 || !aligned16(x)) return false;
    const long long npix = (long long)s.n * s.h * s.w;
    // one block per SM: fewer partial sums to add atomically into the same few outputs
    const unsigned grid = (unsigned)std::min<long long>(sm_count(), (npix + 255) / 256);
    const __nv_bfloat16 *xb = (const __nv_bfloat16*)x, *dyb = (const __nv_bfloat16*)dy;
    if (s.cout == 4 && s.cin == 8) k_wgrad_small<8, 4><<<grid, 256, 0, st>>>(xb, dyb, dw, db, npix);
    else if (s.cout == 4 && s.cin == 16) k_wgrad_small<16, 4><<<grid, 256, 0, st>>>(xb, dyb, dw, db, npix);
    else if (s.cout == 4 && s.cin == 24) k_wgrad_small<24, 4><<<grid, 256, 0, st>>>(xb, dyb, dw, db, npix);
    else if (s.cout == 4 && s.cin == 32) k_wgrad_small<32, 4><<<grid, 256, 0, st>>>(xb, dyb, dw, db, npix);
    else return false;
    *rc = cudaGetLastError() == cudaSuccess ? CLB_NOP_OK : CLB_NOP_ERR_CUDA;
    return true;
}

int status() { return cudaGetLastError() == cudaSuccess ? CLB_NOP_OK : CLB_NOP_ERR_CUDA; }

}  // namespace

// ---------------------------------------------------------------- C ABI
extern "C" int clb_nop_conv_fwd(const void* x, const void* w, const void* wt, const float* bias, void* y,
                                int32_t y_f32, int32_t relu, int32_t n, int32_t h, int32_t wd, int32_t cin,
                                int32_t cout, int32_t taps, void* stream) {
    if (!x || !w || !y || bad_shape(n, h, wd, cin, cout, taps)) return CLB_NOP_ERR_ARG;
    const ConvShape s{n, h, wd, cin, cout, taps};
    const long long M = (long long)n * h * wd, K = (long long)taps * cin;
    int rc;
    if (wt && launch_tma<FWD>(x, wt, bias, nullptr, y, y_f32, relu, s, M, cout, (cudaStream_t)stream, &rc))
        return rc;
    if (wt && launch_tc<FWD>(x, wt, bias, nullptr, y, y_f32, relu, s, M, cout, K, (cudaStream_t)stream, &rc))
        return rc;
    return launch_gemm<FWD>(x, w, bias, nullptr, y, y_f32, relu, s, M, cout, K, 1, (cudaStream_t)stream);
}

extern "C" int clb_nop_conv_dgrad(const void* dy, const void* w, const void* mask, void* dx, int32_t n, int32_t h,
                                  int32_t wd, int32_t cin, int32_t cout, int32_t taps, void* stream) {
    if (!dy || !w || !dx || bad_shape(n, h, wd, cin, cout, taps)) return CLB_NOP_ERR_ARG;
    const ConvShape s{n, h, wd, cin, cout, taps};
    const long long M = (long long)n * h * wd, K = (long long)taps * cout;
    int rc;
    if (launch_tma<DGRAD>(dy, w, nullptr, mask, dx, 0, 0, s, M, cin, (cudaStream_t)stream, &rc)) return rc;
    if (launch_tc<DGRAD>(dy, w, nullptr, mask, dx, 0, 0, s, M, cin, K, (cudaStream_t)stream, &rc)) return rc;
    if (launch_dgrad_small(dy, w, mask, dx, s, (cudaStream_t)stream, &rc)) return rc;
    return launch_gemm<DGRAD>(dy, w, nullptr, mask, dx, 0, 0, s, M, cin, K, 1, (cudaStream_t)stream);
}

extern "C" int clb_nop_conv_wgrad_bias(const void* x, const void* dy, float* dw, float* db, int32_t n, int32_t h,
                                       int32_t wd, int32_t cin, int32_t cout, int32_t taps, int32_t splitk,
                                       void* stream) {
    if (!x || !dy || !dw || bad_shape(n, h, wd, cin, cout, taps)) return CLB_NOP_ERR_ARG;
    const ConvShape s{n, h, wd, cin, cout, taps};
    const cudaStream_t st = (cudaStream_t)stream;
    int rc;
    bool bias_done = false;
    if (launch_wgrad_tma(x, dy, dw, db, s, splitk, st, &rc, &bias_done)) {
        if (rc != CLB_NOP_OK || !db || bias_done) return rc;
        return clb_nop_bias_grad(dy, db, (int64_t)n * h * wd, cout, stream);
    }
    if (launch_wgrad_tc(x, dy, dw, db, s, splitk, st, &rc) || launch_wgrad_small(x, dy, dw, db, s, st, &rc)) return rc;
    if (db) {   // the generic paths: bias gradient in its own pass
        rc = clb_nop_bias_grad(dy, db, (int64_t)n * h * wd, cout, stream);
        if (rc != CLB_NOP_OK) return rc;
        if (launch_wgrad_tc(x, dy, dw, nullptr, s, splitk, st, &rc)) return rc;
    }
    return launch_gemm<WGRAD>(x, dy, nullptr, nullptr, dw, 1, 0, s, (long long)taps * cin, cout, (long long)n * h * wd,
                              splitk, st);
}

extern "C" int clb_nop_conv_wgrad(const void* x, const void* dy, float* dw, int32_t n, int32_t h, int32_t wd,
                                  int32_t cin, int32_t cout, int32_t taps, int32_t splitk, void* stream) {
    return clb_nop_conv_wgrad_bias(x, dy, dw, nullptr, n, h, wd, cin, cout, taps, splitk, stream);
}

extern "C" int clb_nop_bias_grad(const void* dy, float* db, int64_t npix, int32_t c, void* stream) {
    if (!dy || !db || npix < 1 || c < 1) return CLB_NOP_ERR_ARG;
    if (c % 8 == 0 && c / 8 <= BG_THREADS && aligned16(dy)) {
        const long long n8 = npix * (c / 8);
        const unsigned grid = (unsigned)std::min<long long>(BG_BLOCKS, (n8 + BG_THREADS - 1) / BG_THREADS);
        k_bias_grad8<<<grid, BG_THREADS, 0, (cudaStream_t)stream>>>((const uint4*)dy, db, n8, c / 8);
        return status();
    }
    k_bias_grad<<<(unsigned)((npix + 255) / 256), 128, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)dy, db, npix, c);
    return status();
}

extern "C" int clb_nop_pool2(const void* in, void* out, int32_t n, int32_t h, int32_t w, int32_t c, int32_t backward,
                             void* stream) {
    if (!in || !out || n < 1 || h < 2 || w < 2 || c < 1 || (h & 1) || (w & 1)) return CLB_NOP_ERR_ARG;
    const cudaStream_t st = (cudaStream_t)stream;
    if (c % 8 == 0 && aligned16(in) && aligned16(out)) {
        const int G = c / 8;
        if (!backward)
            k_pool2_fwd8<<<nblk((long long)n * (h / 2) * (w / 2) * G), 256, 0, st>>>((const uint4*)in, (uint4*)out, n, h,
                                                                                    w, G);
        else
            k_pool2_bwd8<<<nblk((long long)n * h * w * G), 256, 0, st>>>((const uint4*)in, (uint4*)out, n, h, w, G);
        return status();
    }
    if (!backward)
        k_pool2_fwd<<<nblk((long long)n * (h / 2) * (w / 2) * c), 256, 0, st>>>((const __nv_bfloat16*)in, (__nv_bfloat16*)out, n, h, w, c);
    else
        k_pool2_bwd<<<nblk((long long)n * h * w * c), 256, 0, st>>>((const __nv_bfloat16*)in, (__nv_bfloat16*)out, n, h, w, c);
    return status();
}

extern "C" int clb_nop_up2(const void* in, void* out, int32_t n, int32_t h, int32_t w, int32_t c, int32_t backward,
                           void* stream) {
    if (!in || !out || n < 1 || h < 1 || w < 1 || c < 1) return CLB_NOP_ERR_ARG;
    const cudaStream_t st = (cudaStream_t)stream;
    if (c % 8 == 0 && aligned16(in) && aligned16(out)) {
        const int G = c / 8;
        if (!backward)
            k_up2_fwd8<<<nblk((long long)n * 4 * h * w * G), 256, 0, st>>>((const uint4*)in, (uint4*)out, n, h, w, G);
        else
            k_up2_bwd8<<<nblk((long long)n * h * w * G), 256, 0, st>>>((const uint4*)in, (uint4*)out, n, h, w, G);
        return status();
    }
    if (!backward)
        k_up2_fwd<<<nblk((long long)n * 4 * h * w * c), 256, 0, st>>>((const __nv_bfloat16*)in, (__nv_bfloat16*)out, n, h, w, c);
    else
        k_up2_bwd<<<nblk((long long)n * h * w * c), 256, 0, st>>>((const __nv_bfloat16*)in, (__nv_bfloat16*)out, n, h, w, c);
    return status();
}

extern "C" int clb_nop_concat(void* a, void* b, void* y, int64_t npix, int32_t ca, int32_t cb, int32_t inverse,
                              void* stream) {
    if (!a || !b || !y || npix < 1 || ca < 1 || cb < 1) return CLB_NOP_ERR_ARG;
    if (ca % 8 == 0 && cb % 8 == 0 && aligned16(a) && aligned16(b) && aligned16(y)) {
        k_concat8<<<nblk(npix * ((ca + cb) / 8)), 256, 0, (cudaStream_t)stream>>>((uint4*)a, (uint4*)b, (uint4*)y, npix,
                                                                                  ca / 8, cb / 8, inverse);
        return status();
    }
    k_concat<<<nblk(npix * (ca + cb)), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)a, (const __nv_bfloat16*)b,
                                                                        (__nv_bfloat16*)y, npix, ca, cb, inverse);
    return status();
}

extern "C" int clb_nop_mse(const float* pred, const float* target, const float* wch, int32_t nch, void* grad,
                           float* loss, int64_t n, void* stream) {
    if (!pred || !target || !grad || !loss || n < 1 || nch < 1 || n % nch) return CLB_NOP_ERR_ARG;
    k_mse<<<nblk(n), 256, 0, (cudaStream_t)stream>>>(pred, target, wch, nch, (__nv_bfloat16*)grad, loss, n);
    return status();
}

namespace {
// Bias corrections 1 - b1^t, 1 - b2^t (the power by repeated products, as
// the FP32 moments see it).
void adam_corrections(float b1, float b2, int32_t t, float& c1, float& c2) {
    float p1 = 1.0f, p2 = 1.0f;
    for (int i = 0; i < t && i < 100000; ++i) {
        p1 *= b1;
        p2 *= b2;
    }
    c1 = 1.0f - p1;
    c2 = 1.0f - p2;
}

constexpr int ADAM_SEGS = 32;
struct AdamSegs {
    clb_nop_adam_seg s[ADAM_SEGS];
    int first[ADAM_SEGS + 1];   // first block of each segment
    int n;
};

__global__ void k_adam_multi(const AdamSegs S, float lr, float b1, float b2, float eps, float c1, float c2) {
    int k = 0;
    while (k + 1 < S.n && (int)blockIdx.x >= S.first[k + 1]) ++k;
    const clb_nop_adam_seg& q = S.s[k];
    const long long i = (long long)(blockIdx.x - S.first[k]) * blockDim.x + threadIdx.x;
    if (i >= q.n) return;
    const float gi = q.g[i];
    const float mi = b1 * q.m[i] + (1.0f - b1) * gi;
    const float vi = b2 * q.v[i] + (1.0f - b2) * gi * gi;
    q.m[i] = mi;
    q.v[i] = vi;
    const float wi = q.w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    q.w[i] = wi;
    const __nv_bfloat16 wh = __float2bfloat16(wi);
    if (q.wb) reinterpret_cast<__nv_bfloat16*>(q.wb)[i] = wh;
    if (q.wbt) {
        const int r = (int)(i / q.cols), c = (int)(i - (long long)r * q.cols);
        reinterpret_cast<__nv_bfloat16*>(q.wbt)[(long long)c * q.rows + r] = wh;
    }
}
}  // namespace

extern "C" int clb_nop_adam(float* w, const float* g, float* m, float* v, void* wb, int64_t n, float lr, float b1,
                            float b2, float eps, int32_t t, void* stream) {
    if (!w || !g || !m || !v || n < 1 || t < 1) return CLB_NOP_ERR_ARG;
    float c1, c2;
    adam_corrections(b1, b2, t, c1, c2);
    k_adam<<<nblk(n), 256, 0, (cudaStream_t)stream>>>(w, g, m, v, (__nv_bfloat16*)wb, n, lr, b1, b2, eps, c1, c2);
    return status();
}

extern "C" int clb_nop_adam_multi(const clb_nop_adam_seg* segs, int32_t nseg, float lr, float b1, float b2, float eps,
                                  int32_t t, void* stream) {
    if (!segs || nseg < 1 || t < 1) return CLB_NOP_ERR_ARG;
    for (int k = 0; k < nseg; ++k) {
        const clb_nop_adam_seg& q = segs[k];
        if (!q.w || !q.g || !q.m || !q.v || q.n < 1 || (q.wbt && (q.rows < 1 || q.cols < 1 ||
                                                                   (int64_t)q.rows * q.cols != q.n)))
            return CLB_NOP_ERR_ARG;
    }
    float c1, c2;
    adam_corrections(b1, b2, t, c1, c2);
    for (int k0 = 0; k0 < nseg; k0 += ADAM_SEGS) {
        AdamSegs S;
        S.n = std::min(ADAM_SEGS, nseg - k0);
        long long blocks = 0;
        for (int k = 0; k < S.n; ++k) {
            S.s[k] = segs[k0 + k];
            S.first[k] = (int)blocks;
            blocks += (S.s[k].n + 255) / 256;
        }
        if (blocks >= 2147483647LL) return CLB_NOP_ERR_ARG;
        S.first[S.n] = (int)blocks;
        k_adam_multi<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(S, lr, b1, b2, eps, c1, c2);
        if (cudaGetLastError() != cudaSuccess) return CLB_NOP_ERR_CUDA;
    }
    return CLB_NOP_OK;
}

extern "C" int clb_nop_cast_bf16(const float* x, void* y, int64_t n, void* stream) {
    if (!x || !y || n < 1) return CLB_NOP_ERR_ARG;
    k_cast_bf16<<<nblk(n), 256, 0, (cudaStream_t)stream>>>(x, (__nv_bfloat16*)y, n);
    return status();
}

extern "C" int clb_nop_zero(void* ptr, int64_t bytes, void* stream) {
    if (!ptr || bytes < 0) return CLB_NOP_ERR_ARG;
    return cudaMemsetAsync(ptr, 0, (size_t)bytes, (cudaStream_t)stream) == cudaSuccess ? CLB_NOP_OK : CLB_NOP_ERR_CUDA;
}

namespace {
__global__ void k_add_mask(const __nv_bfloat16* __restrict__ d1, const __nv_bfloat16* __restrict__ d2,
                           const __nv_bfloat16* __restrict__ a, __nv_bfloat16* __restrict__ out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = __bfloat162float(d1[i]);
    if (d2) v += __bfloat162float(d2[i]);
    if (a && !(__bfloat162float(a[i]) > 0.0f)) v = 0.0f;
    out[i] = __float2bfloat16(v);
}
}  // namespace

extern "C" int clb_nop_add_mask(const void* d1, const void* d2, const void* a, void* out, int64_t n, void* stream) {
    if (!d1 || !out || n < 1) return CLB_NOP_ERR_ARG;
    if (n % 8 == 0 && aligned16(d1) && aligned16(out) && (!d2 || aligned16(d2)) && (!a || aligned16(a))) {
        k_add_mask8<<<nblk(n / 8), 256, 0, (cudaStream_t)stream>>>((const uint4*)d1, (const uint4*)d2,
                                                                   (const uint4*)a, (uint4*)out, n / 8);
        return status();
    }
    k_add_mask<<<nblk(n), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)d1, (const __nv_bfloat16*)d2,
                                                          (const __nv_bfloat16*)a, (__nv_bfloat16*)out, n);
    return status();
}

namespace {
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt, int rows,
                                 int cols) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * cols) return;
    const int r = (int)(i / cols), c = (int)(i - (long long)r * cols);
    wt[(long long)c * rows + r] = w[i];
}
}  // namespace

extern "C" int clb_nop_transpose(const void* w, void* wt, int32_t rows, int32_t cols, void* stream) {
    if (!w || !wt || rows < 1 || cols < 1) return CLB_NOP_ERR_ARG;
    k_transpose_bf16<<<nblk((long long)rows * cols), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)w,
                                                                                   (__nv_bfloat16*)wt, rows, cols);
    return status();
}

namespace {
// The tensor-core kernels' failure path on its own: one CTA allocates TMEM
// and waits on an mbarrier that nothing arrives at, with a bound of `limit`
// cycles; the wait expires, the threads agree on the outcome, thread 0 sets
// the time-out flag and warp 0 frees the TMEM -- exactly what k_conv_tc and
// k_wgrad_tc do when their MMAs do not complete in time.  No MMA is issued.
__global__ void __launch_bounds__(TC_THREADS) k_wait_selftest(long long limit) {
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    constexpr uint32_t cols = 32;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&mbar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    bool ok = mbar_wait(smem_u32(&mbar), 0u, limit);   // phase 0 never completes
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0) atomicExch(&g_nop_timeout, 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
}
}  // namespace

extern "C" int clb_nop_wait_selftest(int64_t limit_cycles, void* stream) {
    if (limit_cycles < 1 || limit_cycles > TC_TIMEOUT_CYCLES) return CLB_NOP_ERR_ARG;
    k_wait_selftest<<<1, TC_THREADS, 0, (cudaStream_t)stream>>>((long long)limit_cycles);
    return status();
}

extern "C" int clb_nop_check(void* stream) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return CLB_NOP_ERR_CUDA;
    unsigned int flag = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&flag, g_nop_timeout, sizeof(flag)) != cudaSuccess) return CLB_NOP_ERR_CUDA;
    if (flag && cudaMemcpyToSymbol(g_nop_timeout, &zero, sizeof(zero)) != cudaSuccess) return CLB_NOP_ERR_CUDA;
    return flag ? CLB_NOP_ERR_TIMEOUT : CLB_NOP_OK;
}
