// clb_api.cu -- host side of the C ABI declared in include/clb.h.
//
// Parameter mapping (Sec. 3 and Eqs. 37, 38, 46 of arXiv:2110.05943),
// device memory for the two storage forms (FP64, and FP16 deviations from
// the rest state with FP32 arithmetic), the CUDA-graph step driver, and the
// FP64 reductions for the Nusselt number and the steady-state residual.
#include <cuda.h>             // CUtensorMap (the encoder is fetched from the driver at run time)
#include <cuda_runtime.h>
#include <cudaTypedefs.h>     // PFN_cuTensorMapEncodeTiled

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/clb.h"
#include "clb_kernels.cuh"
#include "clb_reduce.cuh"
#include "clb_tma.cuh"

using namespace clb;

namespace {

constexpr double kCs2 = 1.0 / 3.0;       // D2Q9 c_s^2 (Eq. 15 text)
constexpr int kGraphSteps = 32;          // steps per captured graph (even: same buffer parity)
// Smallest bulk rate for which s3 = 1.2, s4 = 1.8 give a linearly stable
// step (von Neumann threshold 1.19); used when s_b = s_v would fall below it.
constexpr double kSbStable = 1.2;

thread_local std::string g_init_error;


}  // namespace

struct clb_handle {
    clb_params prm{};
    clb_bc bc{};
    clb_lattice lat{};
    KParamsT<double> k64{};       // FP64 form
    KParamsT<float> k32{};        // FP16 forms
    int prec = CLB_F64;
    size_t es = 8;                // bytes per stored distribution value
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int device = 0;
    // distributions, ping-pong: buffer par holds the post-collision values of
    // the last step; par flips every step
    void* f[2] = {nullptr, nullptr};
    void* g[2] = {nullptr, nullptr};
    uint2* rec[2] = {nullptr, nullptr};   // FP16N form: per-node baseline record
    unsigned* seq = nullptr;              // FP16 forms: step counter of each buffer (seeds the rounding)
    int par = 0;
    CoefT<double>* coef = nullptr;   // FP64 form: per-node constants
    float* phi32 = nullptr;          // FP16 forms: porosity (dense) or 1/phi (pitched)
    void* ayg = nullptr;             // a_y - g beta T0 per row (double or float)
    double* scratch = nullptr;       // 4 dense fields (macros, set_fields)
    double* snap = nullptr;          // 3 dense fields (residual reference)
    double* partial = nullptr;       // block partial sums of the reductions
    double* result = nullptr;        // reduction results (device)
    double* host_res = nullptr;      // pinned reduction results
    int n_partial = 0;
    int64_t t = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool graph_failed = false;
    dim3 block, grid;          // one node per thread
    dim3 block2, grid2;        // two nodes per thread (FP16 forms)
    // FP16N form: tensor maps of the TMA-fed interior (per input buffer: f
    // planes, g planes, records; and 1/phi), its tiling, and the wait bound
    CUtensorMap tm_f[2], tm_g[2], tm_r[2], tm_i;
    bool tma_avail = false, tma = false;
    int tma_tiles_x = 0, tma_ntiles = 0, tma_grid = 0;
    unsigned* tma_fail = nullptr;   // device flag set by a CTA whose wait expired
    std::string err;

    AuxT<double> aux64() const { return AuxT<double>{coef, nullptr, nullptr, (const double*)ayg}; }
    AuxT<float> aux32() const {
        return prec == CLB_F16N ? AuxT<float>{nullptr, nullptr, phi32, (const float*)ayg}
                                : AuxT<float>{nullptr, phi32, nullptr, (const float*)ayg};
    }
    template <typename S>
    BufT<S> buf(int i) const { return BufT<S>{(S*)f[i], (S*)g[i], rec[i], seq ? seq + i : nullptr}; }
    const Geo& geo() const { return k64.g; }
    // bytes per node of one stored state (distributions + record)
    size_t node_bytes() const { return 14 * es + (prec == CLB_F16N ? sizeof(uint2) : 0); }
};

static int fail(clb_handle* h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_init_error = buf;
    return code;
}

#define CK(h, call)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            return fail((h), e_ == cudaErrorMemoryAllocation ? CLB_ERR_OOM : CLB_ERR_CUDA,       \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                         \
        }                                                                                        \
    } while (0)

// ------------------------------------------------------------------ defaults
extern "C" void clb_params_default(clb_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->nx = 64;
    p->ny = 64;
    p->precision = CLB_F64;
    p->forchheimer = 1;
    p->shift = 1;
    p->Ra = 1e4;
    p->Da = 1e-2;
    p->Pr = 1.0;
    p->J = 1.0;
    p->Gamma = 1.0;
    p->sigma = 1.0;
    p->Ma = 0.1;
    p->L = 0.0;
    p->nu = 0.0;
    p->dT = 1.0;
    p->T0 = 0.5;
    p->T_init = 0.5;
    p->varpi = 0.25;
    p->s3 = 1.2;
    p->s4 = 1.8;
}

extern "C" void clb_bc_cavity(clb_bc* bc, double Th, double Tc) {
    if (!bc) return;
    std::memset(bc, 0, sizeof *bc);
    for (int s = 0; s < 4; ++s) bc->kind[s] = CLB_WALL;
    bc->thermal[CLB_W] = CLB_ISOTHERMAL;
    bc->T[CLB_W] = Th;
    bc->thermal[CLB_E] = CLB_ISOTHERMAL;
    bc->T[CLB_E] = Tc;
}

// ------------------------------------------------------------------ mapping
// Dimensionless groups -> lattice parameters.
//   Eq. 46:    1/s_v = 1/2 + Ma J L sqrt(3 Pr) / sqrt(Ra)           (nu not given)
//   Sec. 3.1:  1/s_v = 1/2 + J nu / c_s^2                            (nu given)
//   Eq. 15:    nu_e = c_s^2 (1/s_v - 1/2),  nu = nu_e / J
//   Eq. 46:    1/zeta_a = 1/2 + Gamma c_s^2 (1/s_v - 1/2) / (J c_sT^2 Pr)
//   Eq. 37:    alpha_e = c_sT^2 (1/zeta_a - 1/2),  alpha = nu / Pr
//   Eq. 38:    K = Da L^2,  g beta = Ra nu alpha / (dT L^3)
static int map_params(const clb_params* p, clb_lattice* lat, std::string& why) {
    char buf[256];
    auto bad = [&](const char* m) { why = m; return CLB_ERR_ARG; };
    if (p->nx < 1 || p->ny < 1) return bad("nx and ny must be positive");
    if (p->precision != CLB_F64 && p->precision != CLB_F16S && p->precision != CLB_F16N)
        return bad("precision must be CLB_F64, CLB_F16S or CLB_F16N");
    if (!(p->Da > 0) || !(p->Pr > 0) || !(p->J > 0) || !(p->Gamma > 0) || !(p->sigma > 0))
        return bad("Da, Pr, J, Gamma and sigma must be positive");
    if (!(p->Ra >= 0)) return bad("Ra must be >= 0");
    if (!(p->dT > 0)) return bad("dT must be positive");
    if (!(p->varpi > 0 && p->varpi < 1)) return bad("varpi must lie in (0, 1)");
    if (!(p->s3 > 0 && p->s3 < 2) || !(p->s4 > 0 && p->s4 < 2)) return bad("s3 and s4 must lie in (0, 2)");
    const double L = p->L > 0 ? p->L : (double)(p->ny - 1);
    if (!(L > 0)) return bad("characteristic length must be positive (set L or use ny >= 2)");
    double inv_sv;
    if (p->nu > 0) {
        inv_sv = 0.5 + p->J * p->nu / kCs2;
    } else {
        if (!(p->Ra > 0) || !(p->Ma > 0)) return bad("Ra and Ma must be positive when nu is not given");
        inv_sv = 0.5 + p->Ma * p->J * L * std::sqrt(3.0 * p->Pr) / std::sqrt(p->Ra);
    }
    const double nu_e = kCs2 * (inv_sv - 0.5);
    const double nu = nu_e / p->J;
    const double cT2 = 0.5 * p->varpi;
    const double inv_za = 0.5 + p->Gamma * kCs2 * (inv_sv - 0.5) / (p->J * cT2 * p->Pr);
    lat->sv = 1.0 / inv_sv;
    lat->sb = p->sb > 0 ? p->sb : (lat->sv < kSbStable ? kSbStable : lat->sv);
    if (!(lat->sb < 2)) return bad("sb must lie in (0, 2)");
    lat->zeta_a = 1.0 / inv_za;
    lat->nu = nu;
    lat->nu_e = nu_e;
    lat->alpha = nu / p->Pr;
    lat->alpha_e = cT2 * (inv_za - 0.5);
    lat->K = p->Da * L * L;
    lat->gbeta = p->Ra * nu * lat->alpha / (p->dT * L * L * L);
    lat->L = L;
    if (!(lat->sv > 0 && lat->sv < 2) || !(lat->zeta_a > 0 && lat->zeta_a < 2)) {
        std::snprintf(buf, sizeof buf, "relaxation rates out of (0, 2): s_v = %g, zeta_a = %g", lat->sv,
                      lat->zeta_a);
        why = buf;
        return CLB_ERR_ARG;
    }
    return CLB_OK;
}

// Block shapes: 64 x 2 threads for both, one node per thread (FP64) or a
// node pair (FP16: 128 x 2 nodes, each warp a 128-byte line of every FP16
// plane).  Measured at 8192^2 with 7 rest-shifted blocks per SM: F16S
// 78.0 GLUPS with 64-wide blocks, 77.4 with 32 x 4, 76.0 with 16 x 8, 54.6
// with 8 x 16, 78.1 with 128 x 1; F16N 46.7, 46.7, 46.6, 42.5, 46.6.  On
// small grids the blocks shrink (to 64 threads at least) until there are two
// per SM, so a 128^2 cavity is not left on a third of the GPU.
#ifndef CLB_F16_BX
#define CLB_F16_BX 64
#endif
static void shape_blocks(int units, int ny, int bx, int threads, dim3& block, dim3& grid) {
    const long long want = 2LL * 152;
    while (bx > 32 && bx / 2 >= units) bx /= 2;
    int by = threads / bx;
    if (by > ny) by = ny < 1 ? 1 : ny;
    auto count = [&](int a, int b) { return (long long)((units + a - 1) / a) * ((ny + b - 1) / b); };
    while (count(bx, by) < want && bx * by > 64) {
        if (by > 1) by /= 2;
        else bx /= 2;
    }
    block = dim3(bx, by);
    grid = dim3((units + bx - 1) / bx, (ny + by - 1) / by);
}

static void pick_launch(clb_handle* h) {
    const int nx = h->prm.nx, ny = h->prm.ny;
    shape_blocks(nx, ny, CLB_F64_BX, CLB_F64_THREADS, h->block, h->grid);
    shape_blocks((nx + 1) / 2, ny, CLB_F16_BX, 128, h->block2, h->grid2);
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependency on libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
        else
            cudaGetLastError();
    }
    return fn;
}

// Non-swizzled tensor map with zero fill outside the tensor; dims[0] is the
// contiguous dimension, strides[i] the byte stride of dims[i + 1].
static bool encode_map(CUtensorMap* m, CUtensorMapDataType type, const void* base, int rank, const cuuint64_t* dims,
                       const cuuint64_t* strides, const cuuint32_t* box) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint32_t ones[3] = {1, 1, 1};
    return enc(m, type, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps and tiling of the TMA-fed FP16N interior (rows 1 .. ny - 2 in
// tiles of TT_X x TT_Y nodes); false leaves the plain k_step2 path in use.
static bool setup_tma(clb_handle* h) {
    const Geo& G = h->k32.g;
    if (h->prec != CLB_F16N || G.ny < 3 || !h->tma_fail) return false;
    const cuuint64_t px = (cuuint64_t)G.px, ny = (cuuint64_t)G.ny;
    for (int b = 0; b < 2; ++b) {
        const cuuint64_t df[3] = {px, ny, 9}, dg[3] = {px, ny, 5};
        const cuuint64_t sp[2] = {px * 2, (cuuint64_t)G.plane * 2};
        const cuuint32_t bp[3] = {(cuuint32_t)TT_FX, (cuuint32_t)TT_Y, 1};
        const cuuint64_t dr[2] = {px, ny}, sr[1] = {px * 8};
        const cuuint32_t br[2] = {(cuuint32_t)TT_RX, (cuuint32_t)(TT_Y + 2)};
        if (!encode_map(&h->tm_f[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, h->f[b], 3, df, sp, bp) ||
            !encode_map(&h->tm_g[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, h->g[b], 3, dg, sp, bp) ||
            !encode_map(&h->tm_r[b], CU_TENSOR_MAP_DATA_TYPE_UINT64, h->rec[b], 2, dr, sr, br))
            return false;
    }
    const cuuint64_t di[2] = {px, ny}, si[1] = {px * 4};
    const cuuint32_t bi[2] = {(cuuint32_t)TT_IX, (cuuint32_t)(TT_Y + 2)};
    if (!encode_map(&h->tm_i, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, h->phi32, 2, di, si, bi)) return false;
    h->tma_tiles_x = (G.nx + TT_X - 1) / TT_X;
    h->tma_ntiles = h->tma_tiles_x * ((G.ny - 2 + TT_Y - 1) / TT_Y);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms < 1)
        return false;
    h->tma_grid = std::min(h->tma_ntiles, CLB_TT_MINB * sms);   // resident CTAs per SM (launch bounds)
    return h->tma_ntiles > 0;
}

// Reports (and clears) an expired wait of the TMA-fed interior.
static int tma_status(clb_handle* h) {
    if (!h->tma_avail) return CLB_OK;
    unsigned v = 0;
    CK(h, cudaMemcpy(&v, h->tma_fail, sizeof v, cudaMemcpyDeviceToHost));
    if (!v) return CLB_OK;
    CK(h, cudaMemset(h->tma_fail, 0, sizeof v));
    return fail(h, CLB_ERR_TIMEOUT, "a wait for the tile copies of the FP16N step expired; the state is invalid");
}

static void free_all(clb_handle* h) {
    for (int i = 0; i < 2; ++i) {
        if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
        cudaFree(h->f[i]);
        cudaFree(h->g[i]);
        cudaFree(h->rec[i]);
    }
    cudaFree(h->seq);
    cudaFree(h->coef);
    cudaFree(h->phi32);
    cudaFree(h->ayg);
    cudaFree(h->scratch);
    cudaFree(h->snap);
    cudaFree(h->partial);
    cudaFree(h->result);
    if (h->host_res) cudaFreeHost(h->host_res);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
}

// ------------------------------------------------------------------ kernels
template <class P, typename K>
static void step_as(clb_handle* h, cudaStream_t s, const AuxT<typename P::R>& A, const K& kp) {
    using S = typename P::S;
    const BufT<S> in = h->buf<S>(h->par), out = h->buf<S>(1 - h->par);
    const bool sh = h->prm.shift != 0, fo = h->prm.forchheimer != 0;
    // interior tiles, then the wall nodes (see k_step)
    const int tx = (int)h->grid.x, nt = (int)(h->grid.x * h->grid.y);
    const int threads = (int)(h->block.x * h->block.y);
    const unsigned nb = (unsigned)(nt + (wall_count(h->k64.g) + threads - 1) / threads);
    if (sh && fo) k_step<P, true, true><<<nb, h->block, 0, s>>>(in, out, A, kp, tx, nt);
    else if (sh) k_step<P, true, false><<<nb, h->block, 0, s>>>(in, out, A, kp, tx, nt);
    else if (fo) k_step<P, false, true><<<nb, h->block, 0, s>>>(in, out, A, kp, tx, nt);
    else k_step<P, false, false><<<nb, h->block, 0, s>>>(in, out, A, kp, tx, nt);
}

// FP16 forms: two nodes per thread (k_step2), grid over node pairs.
template <class P>
static void step2_as(clb_handle* h, cudaStream_t s, long long limit = TT_LIMIT, int selftest = 0) {
    using S = typename P::S;
    const BufT<S> in = h->buf<S>(h->par), out = h->buf<S>(1 - h->par);
    const AuxT<float> A = h->aux32();
    const bool sh = h->prm.shift != 0, fo = h->prm.forchheimer != 0;
    // pair tiles (interior pairs only), then the edge nodes (see k_step2);
    // with the TMA-fed interior, the pair tiles cover only the rows 0 and
    // ny - 1 of a periodic y
    const Geo& G = h->k32.g;
    const int tx = (int)h->grid2.x;
    int nt = (int)(h->grid2.x * h->grid2.y), outer = 0;
    if constexpr (std::is_same<P, StoreH16N>::value) {
        if (h->tma) {
            const int b = h->par;
            const dim3 gr((unsigned)h->tma_grid), bl(TT_THREADS);
            if (sh && fo)
                k_step2n_tma<true, true><<<gr, bl, TT_SMEM, s>>>(h->tm_f[b], h->tm_g[b], h->tm_r[b], h->tm_i, in, out, A,
                                                                 h->k32, h->tma_tiles_x, h->tma_ntiles, limit, selftest, h->tma_fail);
            else if (sh)
                k_step2n_tma<true, false><<<gr, bl, TT_SMEM, s>>>(h->tm_f[b], h->tm_g[b], h->tm_r[b], h->tm_i, in, out, A,
                                                                  h->k32, h->tma_tiles_x, h->tma_ntiles, limit, selftest, h->tma_fail);
            else if (fo)
                k_step2n_tma<false, true><<<gr, bl, TT_SMEM, s>>>(h->tm_f[b], h->tm_g[b], h->tm_r[b], h->tm_i, in, out, A,
                                                                  h->k32, h->tma_tiles_x, h->tma_ntiles, limit, selftest, h->tma_fail);
            else
                k_step2n_tma<false, false><<<gr, bl, TT_SMEM, s>>>(h->tm_f[b], h->tm_g[b], h->tm_r[b], h->tm_i, in, out, A,
                                                                   h->k32, h->tma_tiles_x, h->tma_ntiles, limit, selftest, h->tma_fail);
            nt = G.wall_y ? 0 : tx;
            outer = 1;
        }
    }
    const int threads = (int)(h->block2.x * h->block2.y);
    const unsigned nb = (unsigned)(nt + (edge_count(G) + threads - 1) / threads);
    if (nb == 0) return;
    if (outer) {
        if (sh && fo) k_step2<P, true, true, true><<<nb, h->block2, 0, s>>>(in, out, A, h->k32, tx, nt);
        else if (sh) k_step2<P, true, false, true><<<nb, h->block2, 0, s>>>(in, out, A, h->k32, tx, nt);
        else if (fo) k_step2<P, false, true, true><<<nb, h->block2, 0, s>>>(in, out, A, h->k32, tx, nt);
        else k_step2<P, false, false, true><<<nb, h->block2, 0, s>>>(in, out, A, h->k32, tx, nt);
    } else {
        if (sh && fo) k_step2<P, true, true><<<nb, h->block2, 0, s>>>(in, out, A, h->k32, tx, nt);
        else if (sh) k_step2<P, true, false><<<nb, h->block2, 0, s>>>(in, out, A, h->k32, tx, nt);
        else if (fo) k_step2<P, false, true><<<nb, h->block2, 0, s>>>(in, out, A, h->k32, tx, nt);
        else k_step2<P, false, false><<<nb, h->block2, 0, s>>>(in, out, A, h->k32, tx, nt);
    }
}

static void launch_step(clb_handle* h, cudaStream_t s) {
    if (h->prec == CLB_F16S) step2_as<StoreH16>(h, s);
    else if (h->prec == CLB_F16N) step2_as<StoreH16N>(h, s);
    else step_as<StoreF64>(h, s, h->aux64(), h->k64);
    h->par = 1 - h->par;
}

template <class P, typename K>
static void macros_as(clb_handle* h, const AuxT<typename P::R>& A, const K& kp, double* r, double* u, double* v,
                      double* T, unsigned long long* bad) {
    using S = typename P::S;
    const BufT<S> in = h->buf<S>(h->par);
    if (h->prm.forchheimer) k_macros<P, true><<<h->grid, h->block, 0, h->stream>>>(in, A, kp, r, u, v, T, bad);
    else k_macros<P, false><<<h->grid, h->block, 0, h->stream>>>(in, A, kp, r, u, v, T, bad);
}

static void launch_macros(clb_handle* h, double* r, double* u, double* v, double* T,
                          unsigned long long* bad = nullptr) {
    if (h->prec == CLB_F16S) macros_as<StoreH16>(h, h->aux32(), h->k32, r, u, v, T, bad);
    else if (h->prec == CLB_F16N) macros_as<StoreH16N>(h, h->aux32(), h->k32, r, u, v, T, bad);
    else macros_as<StoreF64>(h, h->aux64(), h->k64, r, u, v, T, bad);
}

template <class P, typename K>
static void set_fields_as(clb_handle* h, const AuxT<typename P::R>& A, const K& kp, const double* d, long long n) {
    using S = typename P::S;
    k_set_fields<P><<<h->grid, h->block, 0, h->stream>>>(h->buf<S>(0), A, d, d + n, d + 2 * n, d + 3 * n, kp);
}

template <class P, typename K>
static void nusselt_as(clb_handle* h, const AuxT<typename P::R>& A, const K& kp, int nb, int side, double scale) {
    using S = typename P::S;
    k_nusselt_partial<P><<<nb, kRedThreads, 0, h->stream>>>(h->buf<S>(h->par), A, kp, side, scale, h->partial);
}

// Capture kGraphSteps steps starting from buffer parity `par` into an
// executable graph.  Failure is not an error: steps are then launched one by one.
static cudaGraphExec_t capture(clb_handle* h, int par) {
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ex = nullptr;
    const int save = h->par;
    h->par = par;
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        h->par = save;
        cudaGetLastError();
        return nullptr;
    }
    for (int i = 0; i < kGraphSteps; ++i) launch_step(h, h->cap_stream);
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &gr);
    h->par = save;
    if (e != cudaSuccess || !gr) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaGraphInstantiate(&ex, gr, 0) != cudaSuccess) ex = nullptr;
    cudaGraphDestroy(gr);
    cudaGetLastError();
    return ex;
}

// ------------------------------------------------------------------ API
static int set_fields_from_scratch(clb_handle* h);

extern "C" int clb_init(clb_handle** out, const clb_params* p, const double* phi, const double* ay_row,
                        const clb_bc* bc, void* stream) {
    if (!out) return fail(nullptr, CLB_ERR_ARG, "clb_init: output handle pointer is NULL");
    *out = nullptr;
    if (!p || !phi || !bc) return fail(nullptr, CLB_ERR_ARG, "clb_init: params, phi and bc are required");
    clb_lattice lat{};
    std::string why;
    if (map_params(p, &lat, why) != CLB_OK) return fail(nullptr, CLB_ERR_ARG, "clb_init: %s", why.c_str());
    for (int s = 0; s < 4; ++s)
        if (bc->kind[s] != CLB_PERIODIC && bc->kind[s] != CLB_WALL)
            return fail(nullptr, CLB_ERR_ARG, "clb_init: side %d has an unknown kind", s);
    if ((bc->kind[CLB_W] == CLB_WALL) != (bc->kind[CLB_E] == CLB_WALL) ||
        (bc->kind[CLB_S] == CLB_WALL) != (bc->kind[CLB_N] == CLB_WALL))
        return fail(nullptr, CLB_ERR_ARG, "clb_init: opposite sides must both be periodic or both walls");
    const int wall_x = bc->kind[CLB_W] == CLB_WALL, wall_y = bc->kind[CLB_S] == CLB_WALL;
    if ((wall_x && p->nx < 4) || (wall_y && p->ny < 4))
        return fail(nullptr, CLB_ERR_ARG, "clb_init: a walled direction needs at least 4 nodes");
    // size limits first: phi is not read for a grid that is rejected
    if (p->precision != CLB_F64 && (long long)((p->nx + 63) / 64 * 64) * p->ny * 9 > 2147483647LL)
        return fail(nullptr, CLB_ERR_ARG, "clb_init: grid too large for the FP16 forms' 32-bit offsets (9 * ny * pitch >= 2^31)");
    const long long n = (long long)p->nx * p->ny;
    for (long long i = 0; i < n; ++i)
        if (!(phi[i] > 0.0 && phi[i] <= 1.0))
            return fail(nullptr, CLB_ERR_ARG, "clb_init: porosity %g at node %lld is outside (0, 1]", phi[i], i);
    if (ay_row)
        for (int y = 0; y < p->ny; ++y)
            if (!std::isfinite(ay_row[y])) return fail(nullptr, CLB_ERR_ARG, "clb_init: ay_row[%d] is not finite", y);

    clb_handle* h = new (std::nothrow) clb_handle();
    if (!h) return fail(nullptr, CLB_ERR_OOM, "clb_init: out of host memory");
    h->prm = *p;
    h->bc = *bc;
    h->lat = lat;
    h->stream = (cudaStream_t)stream;
    auto bail = [&](int code) {
        g_init_error = h->err;
        free_all(h);
        delete h;
        return code;
    };
#define CKI(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            fail(h, e_ == cudaErrorMemoryAllocation ? CLB_ERR_OOM : CLB_ERR_CUDA, "%s failed: %s", \
                 #call, cudaGetErrorString(e_));                                                  \
            return bail(e_ == cudaErrorMemoryAllocation ? CLB_ERR_OOM : CLB_ERR_CUDA);           \
        }                                                                                         \
    } while (0)
    CKI(cudaGetDevice(&h->device));
    CKI(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));

    h->prec = p->precision;
    const bool half = h->prec != CLB_F64;
    h->es = half ? sizeof(__half) : sizeof(double);
    const int px = (p->nx + 63) / 64 * 64;          // 128 B rows in FP16, 512 B in FP64
    h->lat.pitch = px;
    {
        KParamsT<double> K{};
        K.g.nx = p->nx;
        K.g.ny = p->ny;
        K.g.px = px;
        K.g.plane = (long long)px * p->ny;
        K.g.wall_x = wall_x;
        K.g.wall_y = wall_y;
        for (int s = 0; s < 4; ++s) {
            K.b.uw[s] = bc->u[s];
            K.b.vw[s] = bc->v[s];
            K.b.Tw[s] = bc->T[s];
            K.b.iso[s] = bc->thermal[s] == CLB_ISOTHERMAL;
        }
        K.p.ax = p->ax;
        K.p.gbeta = lat.gbeta;
        K.p.sigma = p->sigma;
        K.p.inv_sigma = 1.0 / p->sigma;
        K.p.cT2 = 0.5 * p->varpi;
        K.p.sv = lat.sv;
        K.p.sp = 0.5 * (lat.sb + lat.sv);
        K.p.sm = 0.5 * (lat.sb - lat.sv);
        K.p.s3 = p->s3;
        K.p.s4 = p->s4;
        K.p.om_a = 1.0 - lat.zeta_a;
        K.p.c6 = (1.0 - 0.5 * p->s3) / 3.0;
        K.p.ca = 1.0 - 0.5 * lat.sv;
        K.p.cb8 = 1.0 - 0.5 * p->s4;
        K.p.sb3 = lat.sb / 3.0;
        K.p.c62 = 2.0 * K.p.c6;
        K.p.s49 = p->s4 / 9.0;
        K.p.hza = 0.5 * lat.zeta_a;
        K.p.hom = 0.5 * (1.0 - lat.zeta_a);
        K.p.hcT2 = 0.5 * K.p.cT2;
        K.nuK = lat.nu / lat.K;
        K.l1c = p->forchheimer ? 0.875 / std::sqrt(150.0 * lat.K) : 0.0;
        K.T0 = p->T0;
        h->k64 = K;
        // FP16 form: same parameters in FP32, and the rest-state offsets the
        // stored deviations are taken from: w_i rho_0 (rho_0 = 1) for f, the
        // D2Q5 equilibrium at rest and T = T0 for g.
        KParamsT<float>& k = h->k32;
        k.g = K.g;
        for (int s = 0; s < 4; ++s) {
            k.b.uw[s] = (float)K.b.uw[s];
            k.b.vw[s] = (float)K.b.vw[s];
            k.b.Tw[s] = (float)K.b.Tw[s];
            k.b.iso[s] = K.b.iso[s];
        }
        const double* pd = &K.p.ax;
        float* pf = &k.p.ax;
        for (size_t i = 0; i < sizeof(PhysT<double>) / sizeof(double); ++i) pf[i] = (float)pd[i];
        k.nuK = (float)K.nuK;
        k.l1c = (float)K.l1c;
        k.T0 = (float)K.T0;
        const double w9[9] = {16.0 / 36, 4.0 / 36, 4.0 / 36, 4.0 / 36, 4.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
        for (int i = 0; i < 9; ++i) {
            k.wf[i] = (float)w9[i];
            k.wfs[i] = k.wf[i] * kDevScale;   // exact (power of two)
        }
        k.wg[0] = (float)((p->sigma - p->varpi) * p->T0);
        for (int i = 1; i < 5; ++i) k.wg[i] = (float)(0.25 * p->varpi * p->T0);
    }
    const Geo& G = h->k64.g;
    pick_launch(h);

    const size_t fbytes = (size_t)G.plane * 9 * h->es;
    const size_t gbytes = (size_t)G.plane * 5 * h->es;
    if (half) {
        // the two buffers' step counters and the TMA wait flag
        CKI(cudaMalloc(&h->seq, 3 * sizeof(unsigned)));
        CKI(cudaMemsetAsync(h->seq, 0, 3 * sizeof(unsigned), h->stream));
        h->tma_fail = h->seq + 2;
    }
    for (int i = 0; i < 2; ++i) {
        CKI(cudaMalloc(&h->f[i], fbytes));
        CKI(cudaMalloc(&h->g[i], gbytes));
        // the pitch padding is never read by the kernels; clear it once
        CKI(cudaMemsetAsync(h->f[i], 0, fbytes, h->stream));
        CKI(cudaMemsetAsync(h->g[i], 0, gbytes, h->stream));
        if (h->prec == CLB_F16N) {
            CKI(cudaMalloc(&h->rec[i], (size_t)G.plane * sizeof(uint2)));
            CKI(cudaMemsetAsync(h->rec[i], 0, (size_t)G.plane * sizeof(uint2), h->stream));
        }
    }
    if (h->prec == CLB_F16S) CKI(cudaMalloc(&h->phi32, (size_t)n * sizeof(float)));
    else if (h->prec == CLB_F16N) {
        CKI(cudaMalloc(&h->phi32, (size_t)G.plane * sizeof(float)));
        CKI(cudaMemsetAsync(h->phi32, 0, (size_t)G.plane * sizeof(float), h->stream));
    } else CKI(cudaMalloc(&h->coef, (size_t)n * sizeof(CoefT<double>)));
    CKI(cudaMalloc(&h->ayg, (size_t)p->ny * (half ? sizeof(float) : sizeof(double))));
    CKI(cudaMalloc(&h->scratch, (size_t)n * 4 * sizeof(double)));
    CKI(cudaMalloc(&h->snap, (size_t)n * 3 * sizeof(double)));
    h->n_partial = reduce_partials(p->nx, p->ny);
    CKI(cudaMalloc(&h->partial, (size_t)h->n_partial * 4 * sizeof(double)));
    CKI(cudaMalloc(&h->result, 8 * sizeof(double)));
    CKI(cudaMallocHost(&h->host_res, 8 * sizeof(double)));

    // a_y per row with g beta T0 folded in: G_y = g beta T + (a_y - g beta T0)
    std::vector<double> ay(p->ny);
    for (int y = 0; y < p->ny; ++y) ay[y] = (ay_row ? ay_row[y] : p->ay) - lat.gbeta * p->T0;
    std::vector<float> ayf(ay.begin(), ay.end());
    if (half)
        CKI(cudaMemcpyAsync(h->ayg, ayf.data(), ayf.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    else
        CKI(cudaMemcpyAsync(h->ayg, ay.data(), ay.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    // per-node constants (FP64 form) or FP32 porosity (FP16 form), staged
    // through the scratch buffer
    CKI(cudaMemcpyAsync(h->scratch, phi, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (half)
        k_phi32<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->scratch, h->phi32, p->nx, p->ny, px,
                                                                      h->prec == CLB_F16N);
    else
        k_coef<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->scratch, (const double*)h->ayg, h->coef,
                                                                     p->nx, n, lat.nu, lat.K, p->ax, lat.gbeta,
                                                                     p->forchheimer);
    CKI(cudaGetLastError());
    CKI(cudaStreamSynchronize(h->stream));

    // start at rest: rho = 1, u = 0, T = T_init, filled on the device
    k_fill4<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->scratch, n, 1.0, 0.0, 0.0, p->T_init);
    CKI(cudaGetLastError());
    int rc = set_fields_from_scratch(h);
    if (rc != CLB_OK) return bail(rc);
    // available, off by default: the F16N step is bound by its arithmetic,
    // not by load latency, and the per-thread kernel measured faster
    h->tma_avail = setup_tma(h);
    h->tma = false;
#undef CKI
    *out = h;
    return CLB_OK;
}

extern "C" int clb_set_fields(clb_handle* h, const double* rho, const double* ux, const double* uy,
                              const double* T) {
    if (!h) return CLB_ERR_ARG;
    if (!rho || !T) return fail(h, CLB_ERR_ARG, "clb_set_fields: rho and T are required");
    const long long n = (long long)h->prm.nx * h->prm.ny;
    for (long long i = 0; i < n; ++i)
        if (!std::isfinite(rho[i]) || !(rho[i] > 0) || !std::isfinite(T[i]) || (ux && !std::isfinite(ux[i])) ||
            (uy && !std::isfinite(uy[i])))
            return fail(h, CLB_ERR_ARG, "clb_set_fields: invalid value at node %lld", i);
    const size_t b = (size_t)n * sizeof(double);
    double* d = h->scratch;
    CK(h, cudaMemcpyAsync(d, rho, b, cudaMemcpyHostToDevice, h->stream));
    if (ux) CK(h, cudaMemcpyAsync(d + n, ux, b, cudaMemcpyHostToDevice, h->stream));
    else CK(h, cudaMemsetAsync(d + n, 0, b, h->stream));
    if (uy) CK(h, cudaMemcpyAsync(d + 2 * n, uy, b, cudaMemcpyHostToDevice, h->stream));
    else CK(h, cudaMemsetAsync(d + 2 * n, 0, b, h->stream));
    CK(h, cudaMemcpyAsync(d + 3 * n, T, b, cudaMemcpyHostToDevice, h->stream));
    return set_fields_from_scratch(h);
}

// Equilibrium state from the four dense fields (rho, ux, uy, T) held in the
// scratch buffer; resets the step counter and the residual reference.
static int set_fields_from_scratch(clb_handle* h) {
    const long long n = (long long)h->prm.nx * h->prm.ny;
    double* d = h->scratch;
    h->par = 0;
    if (h->prec == CLB_F16S) set_fields_as<StoreH16>(h, h->aux32(), h->k32, d, n);
    else if (h->prec == CLB_F16N) set_fields_as<StoreH16N>(h, h->aux32(), h->k32, d, n);
    else set_fields_as<StoreF64>(h, h->aux64(), h->k64, d, n);
    CK(h, cudaGetLastError());
    h->t = 0;
    // residual reference = the new state
    launch_macros(h, nullptr, h->snap, h->snap + n, h->snap + 2 * n);
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(h->stream));
    return CLB_OK;
}

extern "C" int clb_step(clb_handle* h, int64_t n) {
    if (!h) return CLB_ERR_ARG;
    if (n < 0) return fail(h, CLB_ERR_ARG, "clb_step: negative step count");
    int64_t left = n;
    while (left > 0) {
        if (left >= kGraphSteps && !h->graph_failed) {
            if (!h->graph[h->par]) {
                h->graph[h->par] = capture(h, h->par);
                if (!h->graph[h->par]) {
                    h->graph_failed = true;
                    continue;
                }
            }
            CK(h, cudaGraphLaunch(h->graph[h->par], h->stream));   // even count: parity unchanged
            left -= kGraphSteps;
        } else {
            launch_step(h, h->stream);
            CK(h, cudaGetLastError());
            left -= 1;
        }
    }
    h->t += n;
    return CLB_OK;
}

extern "C" int clb_macros_device(clb_handle* h, double* rho, double* ux, double* uy, double* T) {
    if (!h) return CLB_ERR_ARG;
    launch_macros(h, rho, ux, uy, T);
    CK(h, cudaGetLastError());
    return CLB_OK;
}

extern "C" int clb_macros(clb_handle* h, double* rho, double* ux, double* uy, double* T) {
    if (!h) return CLB_ERR_ARG;
    const long long n = (long long)h->prm.nx * h->prm.ny;
    double* d = h->scratch;
    // finiteness is checked on the device (the first bad node's index), not by
    // scanning the copies on the host
    unsigned long long* bad = reinterpret_cast<unsigned long long*>(h->result + 7);
    CK(h, cudaMemsetAsync(bad, 0xFF, sizeof *bad, h->stream));
    launch_macros(h, d, d + n, d + 2 * n, d + 3 * n, bad);
    CK(h, cudaGetLastError());
    double* outs[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k)
        if (outs[k])
            CK(h, cudaMemcpyAsync(outs[k], d + k * n, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(h->host_res + 7, bad, sizeof *bad, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (const int rc = tma_status(h)) return rc;
    unsigned long long first;
    std::memcpy(&first, h->host_res + 7, sizeof first);
    if (first != ~0ULL) return fail(h, CLB_ERR_UNSTABLE, "clb_macros: non-finite value at node %llu", first);
    return CLB_OK;
}

extern "C" int clb_nusselt(clb_handle* h, int32_t side, double* nu) {
    if (!h || !nu) return CLB_ERR_ARG;
    if (side < 0 || side > 3) return fail(h, CLB_ERR_ARG, "clb_nusselt: side must be 0..3");
    const bool along_y = side == CLB_W || side == CLB_E;
    const int len = along_y ? h->prm.ny : h->prm.nx;
    const int depth = along_y ? h->prm.nx : h->prm.ny;
    if (len < 2 || depth < 3) return fail(h, CLB_ERR_ARG, "clb_nusselt: grid too small");
    const int nb = (len + kRedThreads - 1) / kRedThreads;
    if (nb > h->n_partial) return fail(h, CLB_ERR_ARG, "clb_nusselt: too many partials");
    const double scale = -h->lat.L / h->prm.dT / (double)(len - 1);
    if (h->prec == CLB_F16S) nusselt_as<StoreH16>(h, h->aux32(), h->k32, nb, side, scale);
    else if (h->prec == CLB_F16N) nusselt_as<StoreH16N>(h, h->aux32(), h->k32, nb, side, scale);
    else nusselt_as<StoreF64>(h, h->aux64(), h->k64, nb, side, scale);
    k_sum_partials<<<1, kRedThreads, 0, h->stream>>>(h->partial, nb, 1, h->result);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(h->host_res, h->result, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (const int rc = tma_status(h)) return rc;
    *nu = h->host_res[0];
    if (!std::isfinite(*nu)) return fail(h, CLB_ERR_UNSTABLE, "clb_nusselt: non-finite result");
    return CLB_OK;
}

extern "C" int clb_residual(clb_handle* h, double* r_u, double* r_T) {
    if (!h) return CLB_ERR_ARG;
    const long long n = (long long)h->prm.nx * h->prm.ny;
    const int nb = (int)((n + kRedThreads - 1) / kRedThreads);
    const int a = h->par;
    double* d = h->scratch;
    // current macros into scratch, then compare with the snapshot and replace it
    launch_macros(h, nullptr, d, d + n, d + 2 * n);
    const int nbr = nb < h->n_partial ? nb : h->n_partial;
    k_residual_partial<<<nbr, kRedThreads, 0, h->stream>>>(d, h->snap, n, h->partial, nbr);
    k_sum_partials<<<1, kRedThreads, 0, h->stream>>>(h->partial, nbr, 4, h->result);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(h->host_res, h->result, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    (void)a;
    const double du = h->host_res[0], uu = h->host_res[1], dt = h->host_res[2], tt = h->host_res[3];
    if (!std::isfinite(du) || !std::isfinite(uu) || !std::isfinite(dt) || !std::isfinite(tt))
        return fail(h, CLB_ERR_UNSTABLE, "clb_residual: non-finite fields");
    if (r_u) *r_u = uu > 0 ? std::sqrt(du) / std::sqrt(uu) : std::sqrt(du);
    if (r_T) *r_T = tt > 0 ? std::sqrt(dt) / std::sqrt(tt) : std::sqrt(dt);
    return CLB_OK;
}

extern "C" int64_t clb_time(const clb_handle* h) { return h ? h->t : -1; }

extern "C" int clb_lattice_params(const clb_handle* h, clb_lattice* out) {
    if (!h || !out) return CLB_ERR_ARG;
    *out = h->lat;
    return CLB_OK;
}

// Checkpoint layout: 8 int64 header words (magic, version, nx, ny,
// precision, t, step counter of the FP16 forms, 0), then f (9 planes) and
// g (5 planes), each plane ny*nx stored values (FP64, or the FP16
// deviations) without pitch padding.
static const int64_t kMagic = 0x434c42314750554cLL;

extern "C" size_t clb_state_bytes(const clb_handle* h) {
    if (!h) return 0;
    return 8 * sizeof(int64_t) + (size_t)h->prm.nx * h->prm.ny * h->node_bytes();
}

// Copy the 14 distribution planes (and the record plane of the FP16N form)
// between a packed host image and the pitched device buffer `b`.
static int copy_state(clb_handle* h, int b, char* host, bool to_host) {
    const Geo& G = h->geo();
    const int planes = h->prec == CLB_F16N ? 15 : 14;
    size_t off = 0;
    for (int i = 0; i < planes; ++i) {
        const size_t es = i < 14 ? h->es : sizeof(uint2);
        const size_t row = (size_t)h->prm.nx * es, pitch = (size_t)G.px * es;
        char* dev = i < 9 ? (char*)h->f[b] + (size_t)i * G.plane * es
                   : i < 14 ? (char*)h->g[b] + (size_t)(i - 9) * G.plane * es
                            : (char*)h->rec[b];
        if (to_host)
            CK(h, cudaMemcpy2DAsync(host + off, row, dev, pitch, row, h->prm.ny, cudaMemcpyDeviceToHost, h->stream));
        else
            CK(h, cudaMemcpy2DAsync(dev, pitch, host + off, row, row, h->prm.ny, cudaMemcpyHostToDevice, h->stream));
        off += row * h->prm.ny;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return CLB_OK;
}

extern "C" int clb_get_state(clb_handle* h, void* buf, size_t bytes) {
    if (!h || !buf) return CLB_ERR_ARG;
    if (bytes < clb_state_bytes(h)) return fail(h, CLB_ERR_ARG, "clb_get_state: buffer too small");
    unsigned seq = 0;
    if (h->seq) {
        CK(h, cudaMemcpyAsync(&seq, h->seq + h->par, sizeof seq, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    int64_t hdr[8] = {kMagic, 1, h->prm.nx, h->prm.ny, h->prm.precision, h->t, (int64_t)seq, 0};
    std::memcpy(buf, hdr, sizeof hdr);
    return copy_state(h, h->par, (char*)buf + sizeof hdr, true);
}

extern "C" int clb_set_state(clb_handle* h, const void* buf, size_t bytes) {
    if (!h || !buf) return CLB_ERR_ARG;
    if (bytes < clb_state_bytes(h)) return fail(h, CLB_ERR_STATE, "clb_set_state: buffer too small");
    int64_t hdr[8];
    std::memcpy(hdr, buf, sizeof hdr);
    if (hdr[0] != kMagic || hdr[1] != 1 || hdr[2] != h->prm.nx || hdr[3] != h->prm.ny ||
        hdr[4] != h->prm.precision)
        return fail(h, CLB_ERR_STATE, "clb_set_state: checkpoint does not match this simulation");
    h->par = 0;
    if (h->seq) {
        const unsigned seq = (unsigned)hdr[6];
        CK(h, cudaMemcpyAsync(h->seq, &seq, sizeof seq, cudaMemcpyHostToDevice, h->stream));
    }
    const int rc = copy_state(h, 0, (char*)buf + sizeof hdr, false);   // synchronises the stream
    if (rc != CLB_OK) return rc;
    h->t = hdr[5];
    return CLB_OK;
}

extern "C" int clb_sync(clb_handle* h) {
    if (!h) return CLB_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    return tma_status(h);
}

extern "C" int clb_set_tma(clb_handle* h, int32_t enable) {
    if (!h) return CLB_ERR_ARG;
    if (enable && !h->tma_avail)
        return fail(h, CLB_ERR_ARG, "clb_set_tma: the TMA-fed step is not available for this handle");
    if ((enable != 0) != h->tma) {
        // captured graphs hold the other path's launches
        for (int i = 0; i < 2; ++i)
            if (h->graph[i]) {
                cudaGraphExecDestroy(h->graph[i]);
                h->graph[i] = nullptr;
            }
        h->tma = enable != 0;
    }
    return CLB_OK;
}

extern "C" int clb_tma_selftest(clb_handle* h, int64_t limit_cycles) {
    if (!h || limit_cycles < 1) return CLB_ERR_ARG;
    if (!h->tma_avail) return fail(h, CLB_ERR_ARG, "clb_tma_selftest: the TMA-fed step is not available");
    CK(h, cudaStreamSynchronize(h->stream));
    const bool save = h->tma;
    h->tma = true;
    step2_as<StoreH16N>(h, h->stream, (long long)limit_cycles, 1);   // writes the idle buffer; time and parity unchanged
    h->tma = save;
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(h->stream));
    return tma_status(h);
}

extern "C" void clb_destroy(clb_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

// ------------------------------------------------------------------ checks
namespace {
__global__ void k_fp64_special_check(const double* __restrict__ x, long long n, double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    out[4 * i + 0] = clb::recip(v);
    out[4 * i + 1] = 1.0 / v;
    out[4 * i + 2] = clb::sqroot(v);
    out[4 * i + 3] = sqrt(v);
}
}  // namespace

extern "C" int clb_fp64_special_check(const double* x, int64_t n, double* out, void* stream) {
    if (!x || !out || n < 1) return fail(nullptr, CLB_ERR_ARG, "clb_fp64_special_check: bad arguments");
    const long long nb = (n + 255) / 256;
    if (nb > 0x7fffffffLL) return fail(nullptr, CLB_ERR_ARG, "clb_fp64_special_check: n too large");
    k_fp64_special_check<<<(unsigned)nb, 256, 0, (cudaStream_t)stream>>>(x, n, out);
    CK(nullptr, cudaGetLastError());
    return CLB_OK;
}

// Message for clb_last_error(NULL) from entry points without a handle.
void clb_internal_set_error(const char* msg) { g_init_error = msg ? msg : ""; }

extern "C" const char* clb_last_error(const clb_handle* h) {
    return h ? h->err.c_str() : g_init_error.c_str();
}

// ------------------------------------------------------------------ batches
#include "clb_batch.cuh"
