// clb_kernels.cuh -- device code of the coupled porous cascaded LB step.
//
// One thread owns one node.  The fused kernel pulls the 9 + 5 post-collision
// values of the previous step from the node's neighbours (streaming, Eqs. 18
// and 35, as a pull), forms the macroscopic state (Eqs. 20, 22-23, 36, 4),
// collides both lattices (Eqs. 11 and 28) and writes the post-collision
// values back to the node's own slot of the other buffer (ping-pong).  Wall
// nodes rebuild their pre-collision values by non-equilibrium extrapolation
// from the inward neighbour, whose values they pull themselves, so a step is
// one launch with no inter-thread dependency.
//
// The collision is evaluated in "delta" form: with m~ the central moments
// of Eq. 12 and Delta = m~* - m~ from Eq. 11, linearity gives
//   f* = M^-1 N^-1 (m~ + Delta) = f + M^-1 N^-1 Delta,
// so only N m (rows 3..8, Eq. 14), the relaxation increments, N^-1 Delta
// (Eq. A1, with Delta_0 = 0) and M^-1 are needed; every product of the
// dense matrices is expanded by hand into the few multiply-adds its
// non-zero pattern requires.  With s_0 = s_1 = 1 the first-order central
// moments after collision are rho F / 2 (Eq. 11, Eq. 17), and with
// zeta_T = zeta_e = zeta_nu = 1 the thermal moments n~0, n~3, n~4 relax
// straight to Eq. 32, so they are never formed.
//
// Two storage forms share this arithmetic (templated on the real type R):
//   StoreF64 : FP64 distributions, FP64 arithmetic, per-node FP64 constants
//              (1/phi, phi/2, phi nu/K, l1 or 1/(2 l0)) precomputed at init.
//              On GB300 FP64 issues at 2 DFMA/clk/SM, so this form is bound
//              by FP64 instruction throughput, not by HBM; precomputing the
//              constants removes their divisions and square roots.
//   StoreH16 : FP16 storage of each distribution's deviation from its
//              rest-state value (w_i rho_0 for f, the equilibrium at T0 for
//              g), FP32 arithmetic, constants recomputed per node from an
//              FP32 porosity (FP32 is plentiful; bytes are not).  60 B per
//              node update: bound by HBM.  The deviation of the rest
//              population g_0 is O(Delta T), so FP16 quantises T at ~2e-4 of
//              Delta T every step -- too coarse for converged Nusselt numbers.
//   StoreH16N: FP16 storage of each post-collision value's deviation from
//              the local equilibrium f^eq(rho, u; phi), g^eq(T, u) of the
//              node that wrote it, plus that node's (rho - 1, u, T - T0) as
//              four halves.  Writer and reader rebuild the baseline from the
//              same stored halves, so the baseline needs no precision; only
//              the small non-equilibrium remainder is quantised.  FP32
//              arithmetic, 1/phi in FP32; 76 B per node update.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#ifndef CLB_HD
#define CLB_HD __device__ __forceinline__
#endif

namespace clb {

using ::fma;   // keep the float / double overloads visible next to fma(f2, f2, f2)

// Per-node constants derived from the porosity (Eqs. 4, 5, 23) and the
// row's external force.  With them the half force of Eq. 4 is
//   F / 2 = -(hdar + l1 |u|) u + (hgx, hgb T + hgy)
// (G = (a_x, a_y + g beta (T - T0)), hgy carrying a_y - g beta T0).
template <typename R>
struct alignas(8 * sizeof(R)) CoefT {
    R ip;    // 1 / phi
    R l0;    // l0 = (1 + phi nu / (2 K)) / 2 (Eq. 23)
    R l0sq;  // l0^2
    R aux;   // Forchheimer: l1 = phi F_phi / (2 sqrt K); else 1 / (2 l0)
    R hdar;  // phi nu / (2 K): half the Darcy coefficient of Eq. 4
    R hgx;   // phi a_x / 2
    R hgb;   // phi g beta / 2
    R hgy;   // phi (a_y - g beta T0) / 2 of the node's row
};

struct Geo {
    int nx, ny, px;       // grid and row pitch (elements)
    long long plane;      // px * ny
    int wall_x, wall_y;   // W/E resp. S/N are walls
};

template <typename R>
struct BndT {
    R uw[4], vw[4], Tw[4];
    int iso[4];
};

template <typename R>
struct PhysT {
    R ax, gbeta, sigma, inv_sigma, cT2;   // a_x, g*beta, sigma, 1/sigma, c_sT^2
    R sv, s3, s4, om_a;                   // relaxation rates, om_a = 1 - zeta_alpha
    R sp, sm;                             // (s_b + s_v)/2, (s_b - s_v)/2: (k20, k02) block of Eq. 15
    R c6;                                 // (1 - s3/2) / 3  (Eq. 11 rows 6, 7 with Eq. 17)
    R ca, cb8;                            // unit-shift variant: 1 - s_v/2, 1 - s4/2
    R sb3, c62, s49;                      // s_b / 3, 2 c6, s4 / 9
    R hza, hom, hcT2;                     // zeta_a / 2, (1 - zeta_a) / 2, c_sT^2 / 2
};

template <typename R>
struct KParamsT {
    Geo g;
    BndT<R> b;
    PhysT<R> p;
    R nuK;        // nu / K       (FP16 forms: per-node constants from phi)
    R l1c;        // 0.875 / sqrt(150 K): l1 = l1c / sqrt(phi)
    R T0;         // reference temperature (baseline record of the FP16N form)
    R wf[9];      // rest-state offsets of the stored distributions (FP16 form)
    R wg[5];
    R wfs[9];     // wf * 2^12 (the stored scale)
};

// Pointers that are not distributions: per-node constants (FP64 form),
// porosity (FP16 rest-shifted form, dense) or 1/phi (FP16 equilibrium-shifted
// form, pitched like the planes), and a_y - g beta T0 per row.
template <typename R>
struct AuxT {
    const CoefT<R>* coef;
    const float* phi;
    const float* ip;
    const R* ayg;
};

// One ping-pong buffer: distribution planes, and for the equilibrium-shifted
// FP16 form the per-node baseline record (rho - 1, u_x, u_y, T - T0) as four
// halves.
template <typename S>
struct BufT {
    S* f;
    S* g;
    uint2* rec;
    unsigned* seq;   // FP16 forms: steps taken to reach the state this buffer holds (seeds the rounding)
};

template <typename S>
__host__ __device__ inline BufT<const S> as_const(const BufT<S>& b) {
    return BufT<const S>{b.f, b.g, b.rec, b.seq};
}

// ---------------------------------------------------------------- rounding
// The FP16 forms store their values with unbiased stochastic rounding:
// round-to-nearest of a value that depends on the state is a systematic
// error that the time march accumulates (it acts as a steady heat source),
// whereas randomised rounding leaves zero-mean noise.  sm_100-family GPUs
// round stochastically in hardware: cvt.rs.f16x2.f32 adds 13 random bits
// below the 10 kept mantissa bits (the 13 that FP32 -> FP16 drops) and
// truncates, so a value is rounded away from zero with probability equal
// to its dropped fraction -- the expected stored value equals the FP32
// value exactly.  Its first source goes to the upper half and draws on bits
// 16..28 of the random word, the second on bits 0..12 (checked on the GPU).
// The words come from the 32-bit integer mixer "lowbias32" (C. Wellons'
// hash-prospector) keyed by the node's plane offset and the buffer's step
// counter: h0 = mix(node, step), h1 = an odd multiple of a second mix, and
// value k of a node (pair) uses h0 + k h1 (a Weyl sequence: every word,
// and each 13-bit field of it, is uniform).  Runs stay deterministic and
// bit-reproducible.
CLB_HD uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

struct Dither {
    uint32_t h0, h1;   // value k uses the word h0 + k h1
};

CLB_HD Dither dither_for(uint32_t node, uint32_t seq) {
    Dither d;
    d.h0 = mix32(node * 0x9E3779B1U ^ mix32(seq + 0x632BE5ABU));
    d.h1 = ((d.h0 ^ (d.h0 >> 15)) * 0x85EBCA77U) | 1U;
    return d;
}

CLB_HD uint32_t dword(const Dither& d, int k) { return d.h0 + (uint32_t)k * d.h1; }

// lo -> .x (bits 0..15), hi -> .y, stochastically rounded with the random word r.
CLB_HD __half2 sr_half2(float lo, float hi, uint32_t r) {
    uint32_t v;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(v) : "f"(hi), "f"(lo), "r"(r));
    return *reinterpret_cast<const __half2*>(&v);
}

CLB_HD __half sr_half(float v, uint32_t r) { return __low2half(sr_half2(v, 0.0f, r)); }

// Stored FP16 values are the deviations times 2^12 (exact): most
// deviations of the equilibrium-shifted form lie below FP16's smallest
// normal number (6.1e-5), where FP16 has a fixed absolute spacing;
// scaled, everything above 1.5e-8 keeps FP16's full relative precision.
// The largest storable deviation is 16.
constexpr float kDevScale = 4096.0f, kDevInv = 1.0f / 4096.0f;

__device__ __forceinline__ int wrap_lo(int a, int n) { return a < 0 ? a + n : a; }
__device__ __forceinline__ int wrap_hi(int a, int n) { return a >= n ? a - n : a; }

// Plane offsets of the values streaming into (x, y): f_i(x) = f*_i(x - e_i)
// (Eqs. 18 and 35), with periodic wrap (walled directions never wrap for
// the nodes that pull).  I = long long for FP64 buffers, int for FP16 ones
// (clb_init checks that every FP16 offset fits).
template <typename I>
__device__ __forceinline__ void sources(const Geo& G, int x, int y, I (&o)[9]) {
    const int xm = wrap_lo(x - 1, G.nx), xp = wrap_hi(x + 1, G.nx);
    const int ym = wrap_lo(y - 1, G.ny), yp = wrap_hi(y + 1, G.ny);
    const I r0 = (I)y * G.px, rm = (I)ym * G.px, rp = (I)yp * G.px;
    o[0] = r0 + x;
    o[1] = r0 + xm;
    o[2] = rm + x;
    o[3] = r0 + xp;
    o[4] = rp + x;
    o[5] = rm + xm;
    o[6] = rm + xp;
    o[7] = rp + xp;
    o[8] = rp + xm;
}

// ---------------------------------------------------------------- packed FP32
// Two FP32 lanes in one 64-bit register, operated on by the f32x2 forms of
// add / sub / mul / fma (sm_100 and later): the FP16 forms run two nodes per
// thread through the same templated arithmetic with R = f2, halving the
// FP32 instructions issued per node.
struct f2 {
    unsigned long long v;
    f2() = default;
    __device__ __forceinline__ explicit f2(double c) { v = pack((float)c, (float)c); }
    static __device__ __forceinline__ unsigned long long pack(float a, float b) {
        unsigned long long r;
        asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
        return r;
    }
    static __device__ __forceinline__ f2 make(float a, float b) {
        f2 r;
        r.v = pack(a, b);
        return r;
    }
    __device__ __forceinline__ float lo() const { return __uint_as_float((unsigned)(v & 0xffffffffull)); }
    __device__ __forceinline__ float hi() const { return __uint_as_float((unsigned)(v >> 32)); }
};

__device__ __forceinline__ f2 operator+(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 operator-(f2 a) {
    f2 r;
    r.v = a.v ^ 0x8000000080000000ull;   // flip both sign bits
    return r;
}
__device__ __forceinline__ f2& operator+=(f2& a, f2 b) { return a = a + b; }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

// Reciprocal and square root.
// FP64: the hardware estimates rcp.approx.ftz.f64 / rsqrt.approx.ftz.f64
// (relative error ~1e-6, measured) refined by one third-order Newton-Raphson
// step (Newton's iteration with its second-order correction term, Householder
// order 2):
//   1/x       = r (1 + e + e^2),              e = 1 - x r,
//   1/sqrt(s) = y (1 + e/2 + 3 e^2 / 8),      e = 1 - s y^2,   sqrt(s) = s / sqrt(s).
// The error after the step is O(e^3) ~ 1e-18: the results are within 2 ulp
// of the correctly rounded ones (checked on the GPU against CUDA's IEEE
// division and sqrt).  They cost 3 and 6 FP64-pipe instructions against
// ~6 and ~9.5 for the IEEE routines -- the FP64 step is bound by that pipe.
// sqroot needs s > 0 (rsqrt(0) is infinite): callers add 1e-300, which
// changes no square root of a representable velocity.
// FP32: the hardware approximations (relative error ~1e-7, far below the
// FP16 storage resolution of the forms that compute in FP32).
CLB_HD double recip(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}
CLB_HD double sqroot(double s) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(s));
    const double e = fma(-s, y * y, 1.0);
    const double sy = s * y;
    return fma(sy * e, fma(0.375, e, 0.5), sy);
}
// Offset that keeps the argument of sqroot positive (FP64 only).
template <typename R>
CLB_HD R sqrt_guard() { return R(0); }
template <>
CLB_HD double sqrt_guard<double>() { return 1e-300; }

__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ float sqroot(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ f2 recip(f2 x) { return f2::make(recip(x.lo()), recip(x.hi())); }
__device__ __forceinline__ f2 sqroot(f2 x) { return f2::make(sqroot(x.lo()), sqroot(x.hi())); }

// Raw moments of Eq. 12, M f, with the shared partial sums of M's rows.
template <typename R>
struct Mom9T {
    R rho, jx, jy, k20, k02, k11, k21, k12, k22;
};

template <typename R>
CLB_HD Mom9T<R> moments9(const R (&f)[9]) {
    const R a = f[5] + f[7], b = f[6] + f[8];
    const R c = f[5] - f[7], d = f[6] - f[8];
    const R s13 = f[1] + f[3], s24 = f[2] + f[4];
    Mom9T<R> k;
    k.k22 = a + b;
    k.k11 = a - b;
    k.k21 = c + d;
    k.k12 = c - d;
    k.k20 = s13 + k.k22;
    k.k02 = s24 + k.k22;
    k.jx = (f[1] - f[3]) + k.k12;
    k.jy = (f[2] - f[4]) + k.k21;
    k.rho = (f[0] + s13) + (s24 + k.k22);
    return k;
}

// Macroscopic velocity by Eqs. 22-23 and half the force of Eq. 4 at a node
// with density rho, momentum j = sum e f and temperature T:
//   v = j / rho + phi G / 2,  u = v / (l0 + sqrt(l0^2 + l1 |v|)),
//   F / 2 = -(phi nu / (2 K) + l1 |u|) u + phi G / 2
// (phi F_phi / sqrt(K) |u| u / 2 = l1 |u| u by the definition of l1).
template <typename R, bool FORCH>
CLB_HD void macro_velocity(R rho, R jx, R jy, R T, const CoefT<R>& c, R& X, R& Y, R& hFx, R& hFy) {
    const R irho = recip(rho);
    const R hGy = fma(c.hgb, T, c.hgy);
    const R vx = fma(jx, irho, c.hgx), vy = fma(jy, irho, hGy);
    R hcF;
    if (FORCH) {
        const R vm = sqroot(fma(vx, vx, fma(vy, vy, sqrt_guard<R>())));
        const R inv = recip(c.l0 + sqroot(fma(c.aux, vm, c.l0sq)));
        X = vx * inv;
        Y = vy * inv;
        hcF = fma(c.aux, vm * inv, c.hdar);      // (phi nu/K + phi F_phi/sqrt(K) |u|) / 2
    } else {
        X = vx * c.aux;
        Y = vy * c.aux;
        hcF = c.hdar;
    }
    hFx = fma(-hcF, X, c.hgx);
    hFy = fma(-hcF, Y, hGy);
}

// Porous flow equilibrium f^eq = M^-1 m^eq (Eq. 19).
template <typename R>
CLB_HD void feq9(R rho, R X, R Y, R ip, R (&fe)[9]) {
    const R X2 = X * X, Y2 = Y * Y;
    const R r3 = rho * R(1.0 / 3.0);
    const R m1 = rho * X, m2 = rho * Y;
    const R m3 = fma(m1 * ip, X, r3);
    const R m4 = fma(m2 * ip, Y, r3);
    const R m5 = m1 * Y * ip;
    const R m6 = fma(m1 * ip, X * Y, r3 * Y);
    const R m7 = fma(m2 * ip, X * Y, r3 * X);
    const R m8 = rho * R(1.0 / 9.0) + r3 * ip * (X2 + Y2) + rho * X2 * Y2 * ip * ip;
    fe[0] = rho - m3 - m4 + m8;
    fe[1] = R(0.5) * (m1 + m3 - m7 - m8);
    fe[2] = R(0.5) * (m2 + m4 - m6 - m8);
    fe[3] = R(0.5) * (-m1 + m3 + m7 - m8);
    fe[4] = R(0.5) * (-m2 + m4 + m6 - m8);
    fe[5] = R(0.25) * (m5 + m6 + m7 + m8);
    fe[6] = R(0.25) * (-m5 + m6 - m7 + m8);
    fe[7] = R(0.25) * (m5 - m6 - m7 + m8);
    fe[8] = R(0.25) * (-m5 - m6 + m7 + m8);
}

// Thermal equilibrium g^eq = M_T^-1 n^eq (Eq. 33; equals Eq. 34).
template <typename R>
CLB_HD void geq5(R T, R X, R Y, R sigma, R cT2, R (&ge)[5]) {
    const R n1 = X * T, n2 = Y * T;
    const R n3 = fma(X, n1, cT2 * T), n4 = fma(Y, n2, cT2 * T);
    ge[0] = sigma * T - n3 - n4;
    ge[1] = R(0.5) * (n1 + n3);
    ge[2] = R(0.5) * (n2 + n4);
    ge[3] = R(0.5) * (n3 - n1);
    ge[4] = R(0.5) * (n4 - n2);
}

// Flow collision (Eq. 11) in delta form; see the file comment.  Result:
// the raw-moment increments r = N^-1 Delta (Eq. A1; r_0 = 0), which
// apply9 turns into f* = f + M^-1 r.  Inputs: the raw moments k of the
// pre-collision f, rho, u = (X, Y), half the force hF = F / 2, 1/phi.
template <typename R>
struct Incr9T {
    R r1, r2, r3, r4, r5, r6, r7, r8;
};

template <typename R, bool SHIFT>
CLB_HD Incr9T<R> collide9_incr(const Mom9T<R>& k, R rho, R X, R Y, R hFx, R hFy, R ip, const PhysT<R>& P) {
    const R rhFx = rho * hFx, rhFy = rho * hFy;                  // S~1 / 2, S~2 / 2 (Eq. 17)
    const R px = fma(rho, X, -k.jx), py = fma(rho, Y, -k.jy);   // -(k~10), -(k~01)
    const R X2 = X * X, Y2 = Y * Y, XY = X * Y;
    const R X2p = X + X, Y2p = Y + Y;
    Incr9T<R> r;
    r.r1 = px + rhFx;                                           // Delta_1 = -k~10 + S~1 / 2 (s_1 = 1)
    r.r2 = py + rhFy;
    const R D1 = r.r1, D2 = r.r2;
    if (SHIFT) {
        // central moments m~3..m~8 = rows 3..8 of N (Eq. 14) times m
        const R ipX = ip * X, ipY = ip * Y;
        const R t = px - k.jx, tp = py - k.jy;        // rho X - 2 jx, rho Y - 2 jy
        const R Xjy = X * k.jy, Yjx = Y * k.jx;
        const R c3 = fma(ipX, t, k.k20);
        const R c4 = fma(ipY, tp, k.k02);
        const R c5 = fma(ip, fma(Y, px, -Xjy), k.k11);
        const R w = fma(-Y, t, Xjy);
        const R c6 = fma(ipX, w, fma(-Y, k.k20, fma(-X2p, k.k11, k.k21)));
        const R wp = fma(-X, tp, Yjx);
        const R c7 = fma(ipY, wp, fma(-X, k.k02, fma(-Y2p, k.k11, k.k12)));
        R A = Y2 * k.k20;
        A = fma(X2, k.k02, A);
        A = fma(R(4) * XY, k.k11, A);
        A = fma(-Y2p, k.k21, A);
        A = fma(-X2p, k.k12, A);
        const R ipXY = ip * XY;
        A = fma(-ipXY, w + Xjy, A);
        const R c8 = fma(ip, A, k.k22);
        // increments of Eq. 11 (Lambda of Eq. 15, s_0 = s_1 = 1); the
        // (k20, k02) block relaxes towards rho / 3 each:
        // D3 = s+ (rho/3 - c3) + s- (rho/3 - c4) = s_b rho / 3 - s+ c3 - s- c4
        const R sbr = P.sb3 * rho;
        const R D3 = fma(-P.sp, c3, fma(-P.sm, c4, sbr));
        const R D4 = fma(-P.sp, c4, fma(-P.sm, c3, sbr));
        const R D5 = -P.sv * c5;
        const R D6 = fma(-P.s3, c6, P.c62 * rhFy);   // + (1 - s3/2) rho Fy / 3
        const R D7 = fma(-P.s3, c7, P.c62 * rhFx);
        const R D8 = fma(P.s49, rho, -P.s4 * c8);     // s4 (rho/9 - c8)
        // back to raw moments: N^-1 Delta (Eq. A1), Delta_0 = 0
        const R ipX2 = ipX + ipX, ipY2 = ipY + ipY;
        const R XD2 = X * D2;
        r.r3 = fma(ipX2, D1, D3);
        r.r4 = fma(ipY2, D2, D4);
        r.r5 = fma(ipY, D1, fma(ipX, D2, D5));
        r.r6 = fma(ipX, fma(Y2p, D1, XD2), fma(Y, D3, fma(X2p, D5, D6)));
        r.r7 = fma(ipY, fma(Y, D1, X2p * D2), fma(X, D4, fma(Y2p, D5, D7)));
        R B = Y2 * D3;
        B = fma(X2, D4, B);
        B = fma(R(4) * XY, D5, B);
        B = fma(Y2p, D6, B);
        B = fma(X2p, D7, B);
        B = fma((ipXY + ipXY), fma(Y, D1, XD2), B);
        r.r8 = fma(ip, B, D8);
    } else {
        // unit shift: relax raw moments towards Eq. 19's m^eq with Eq. 19's S
        const R rFx = rhFx + rhFx, rFy = rhFy + rhFy;
        const R r3 = rho * R(1.0 / 3.0), r9 = rho * R(1.0 / 9.0);
        const R ipr = ip * rho;
        const R meq3 = fma(ipr * X, X, r3), meq4 = fma(ipr * Y, Y, r3);
        const R meq5 = ipr * XY;
        const R meq6 = fma(ipr * X2, Y, r3 * Y), meq7 = fma(ipr * Y2, X, r3 * X);
        const R meq8 = r9 + r3 * ip * (X2 + Y2) + ipr * ip * X2 * Y2;
        const R S3 = R(2) * ip * X * rFx, S4 = R(2) * ip * Y * rFy;
        const R S5 = ip * fma(X, rFy, Y * rFx);
        const R S6 = fma(ip, fma(X2, rFy, R(2) * XY * rFx), rFy * R(1.0 / 3.0));
        const R S7 = fma(ip, fma(Y2, rFx, R(2) * XY * rFy), rFx * R(1.0 / 3.0));
        const R S8 = R(2.0 / 3.0) * ip * fma(X, rFx, Y * rFy) + R(2) * ip * ip * XY * fma(Y, rFx, X * rFy);
        // (k20, k02) block: -Lambda_b (m - m^eq) + (I - Lambda_b / 2) S
        const R d3 = k.k20 - meq3, d4 = k.k02 - meq4;
        r.r3 = -fma(P.sp, d3, P.sm * d4) + S3 - R(0.5) * fma(P.sp, S3, P.sm * S4);
        r.r4 = -fma(P.sm, d3, P.sp * d4) + S4 - R(0.5) * fma(P.sm, S3, P.sp * S4);
        r.r5 = fma(-P.sv, k.k11 - meq5, P.ca * S5);
        r.r6 = fma(-P.s3, k.k21 - meq6, R(3) * P.c6 * S6);
        r.r7 = fma(-P.s3, k.k12 - meq7, R(3) * P.c6 * S7);
        r.r8 = fma(-P.s4, k.k22 - meq8, P.cb8 * S8);
    }
    return r;
}

// f* = f + M^-1 r with r = (0, r1, ..., r8) (Eq. 13's M inverted).
template <typename R>
CLB_HD void apply9(R (&f)[9], const Incr9T<R>& r) {
    const R pa = r.r3 - r.r8, qa = r.r1 - r.r7;
    const R pb = r.r4 - r.r8, qb = r.r2 - r.r6;
    const R u1 = r.r8 + r.r5, u2 = r.r8 - r.r5, v1 = r.r6 + r.r7, v2 = r.r6 - r.r7;
    f[0] = (f[0] - pa) - r.r4;                  // f0 + r8 - r3 - r4
    f[1] = fma(R(0.5), pa + qa, f[1]);
    f[3] = fma(R(0.5), pa - qa, f[3]);
    f[2] = fma(R(0.5), pb + qb, f[2]);
    f[4] = fma(R(0.5), pb - qb, f[4]);
    f[5] = fma(R(0.25), u1 + v1, f[5]);
    f[7] = fma(R(0.25), u1 - v1, f[7]);
    f[6] = fma(R(0.25), u2 + v2, f[6]);
    f[8] = fma(R(0.25), u2 - v2, f[8]);
}

template <typename R, bool SHIFT>
CLB_HD void collide9(R (&f)[9], const Mom9T<R>& k, R rho, R X, R Y, R hFx, R hFy, R ip, const PhysT<R>& P) {
    apply9(f, collide9_incr<R, SHIFT>(k, rho, X, Y, hFx, hFy, ip, P));
}

// Temperature collision (Eq. 28) with zeta_T = zeta_e = zeta_nu = 1:
// g* = M_T^-1 N_T^-1 n~*, n~* = (sigma T, (1 - zeta_a) n~1, (1 - zeta_a) n~2,
// c_sT^2 T, c_sT^2 T), where n~1 = n1 - u_x T (Eq. 31 with sigma T = n0).
// Back-shifting (N_T^-1) gives n1* = u_x T + n~1* = zeta_a u_x T + (1 - zeta_a) n1
// and n3* = u_x^2 T + 2 u_x n~1* + c_sT^2 T = (c_sT^2 - u_x^2) T + 2 u_x n1*.
// The unit-shift variant relaxes the raw moments towards Eq. 33 instead:
// n1* as above, n3* = (c_sT^2 + u_x^2) T.  M_T^-1 then gives
// g0 = n0 - n3* - n4*, g1,3 = (n3* +- n1*) / 2, g2,4 = (n4* +- n2*) / 2;
// the halves h = n* / 2 are formed directly.  Only n0, g1 - g3 and g2 - g4
// of the pre-collision g are used.
template <typename R, bool SHIFT>
CLB_HD void collide5(R (&g)[5], R n0, R T, R X, R Y, const PhysT<R>& P) {
    const R hzT = P.hza * T;
    const R h1 = fma(P.hom, g[1] - g[3], hzT * X);
    const R h2 = fma(P.hom, g[2] - g[4], hzT * Y);
    const R X2 = X * X, Y2 = Y * Y;
    R h3, h4;
    if (SHIFT) {
        h3 = fma(X + X, h1, T * fma(R(-0.5), X2, P.hcT2));
        h4 = fma(Y + Y, h2, T * fma(R(-0.5), Y2, P.hcT2));
    } else {
        h3 = T * fma(R(0.5), X2, P.hcT2);
        h4 = T * fma(R(0.5), Y2, P.hcT2);
    }
    g[0] = fma(R(-2), h3 + h4, n0);
    g[1] = h3 + h1;
    g[3] = h3 - h1;
    g[2] = h4 + h2;
    g[4] = h4 - h2;
}

// Rest-centred thermal representation (the FP16N form).  With q_i(u) =
// g^eq_i(1, u) and the rest state g_rest = T0 q(0), a form that carries
// g~ = g - g_rest and T~ = T - T0 never rounds an O(0.1..0.4) distribution
// in FP32 (that rounding, state-correlated and integrated over long thermal
// times, biased the steady temperature).  Exact identities used:
//   g^eq_i(T, u) - T0 q_i(0) = T~ q_i(u) + T0 (q_i(u) - q_i(0))
//     = T~ (sigma - 2 cT2) - T |u|^2                       (i = 0)
//     = (T~ cT2 + T u_d (u_d +- 1)) / 2                     (i = 1..4, d = x, y)
// and, the thermal collision being linear in (g, n0, T) at fixed u,
//   collide(g~ + g_rest, n0~ + sigma T0, T~ + T0) - g_rest
//     = collide(g~, n0~, T~) + T0 k(u),
//   k_0 = -b |u|^2,  k_{1,3} = (b X^2 +- a X) / 2,  k_{2,4} = (b Y^2 +- a Y) / 2,
// a = zeta_a, b = 1 - 2 (1 - zeta_a) with the shift and 1 without it.
template <int I, typename R>
CLB_HD R geqc_comp(R Tt, R X, R Y, R sigma, R cT2, R T0) {
    if (I == 0) return fma(Tt, sigma - R(2) * cT2, -(Tt + T0) * fma(X, X, Y * Y));
    const R u = (I == 1 || I == 3) ? X : Y;
    const R hT = fma(Tt, R(0.5), R(0.5) * T0);     // T / 2
    return fma(Tt, R(0.5) * cT2, hT * (u * (u + R((I == 1 || I == 2) ? 1.0 : -1.0))));
}

template <typename R>
CLB_HD void geq5c(R Tt, R X, R Y, R sigma, R cT2, R T0, R (&ge)[5]) {
    ge[0] = geqc_comp<0>(Tt, X, Y, sigma, cT2, T0);
    ge[1] = geqc_comp<1>(Tt, X, Y, sigma, cT2, T0);
    ge[2] = geqc_comp<2>(Tt, X, Y, sigma, cT2, T0);
    ge[3] = geqc_comp<3>(Tt, X, Y, sigma, cT2, T0);
    ge[4] = geqc_comp<4>(Tt, X, Y, sigma, cT2, T0);
}

template <typename R, bool SHIFT>
CLB_HD void collide5_centred(R (&g)[5], R n0t, R Tt, R X, R Y, R T0, const PhysT<R>& P) {
    collide5<R, SHIFT>(g, n0t, Tt, X, Y, P);
    const R a = R(1) - P.om_a, b = SHIFT ? fma(R(-2), P.om_a, R(1)) : R(1);
    const R bX2 = b * X * X, bY2 = b * Y * Y, aX = a * X, aY = a * Y, hT0 = R(0.5) * T0;
    g[0] = fma(-T0, bX2 + bY2, g[0]);
    g[1] = fma(hT0, bX2 + aX, g[1]);
    g[3] = fma(hT0, bX2 - aX, g[3]);
    g[2] = fma(hT0, bY2 + aY, g[2]);
    g[4] = fma(hT0, bY2 - aY, g[4]);
}

// Half the force of Eq. 4 at a node whose velocity is imposed (wall nodes).
template <typename R, bool FORCH>
CLB_HD void force_at(R X, R Y, R T, const CoefT<R>& c, R& hFx, R& hFy) {
    R hcF = c.hdar;
    if (FORCH) hcF = fma(c.aux, sqroot(fma(X, X, fma(Y, Y, sqrt_guard<R>()))), c.hdar);
    hFx = fma(-hcF, X, c.hgx);
    hFy = fma(-hcF, Y, fma(c.hgb, T, c.hgy));
}

template <typename R>
__device__ __forceinline__ R sum5(const R (&v)[5]) {
    return ((v[0] + v[1]) + (v[2] + v[3])) + v[4];
}

// Model parameters for the paired path.
__device__ __forceinline__ PhysT<f2> splat(const PhysT<float>& p) {
    PhysT<f2> q;
    q.ax = f2(p.ax);
    q.gbeta = f2(p.gbeta);
    q.sigma = f2(p.sigma);
    q.inv_sigma = f2(p.inv_sigma);
    q.cT2 = f2(p.cT2);
    q.sv = f2(p.sv);
    q.s3 = f2(p.s3);
    q.s4 = f2(p.s4);
    q.om_a = f2(p.om_a);
    q.sp = f2(p.sp);
    q.sm = f2(p.sm);
    q.c6 = f2(p.c6);
    q.ca = f2(p.ca);
    q.cb8 = f2(p.cb8);
    q.sb3 = f2(p.sb3);
    q.c62 = f2(p.c62);
    q.s49 = f2(p.s49);
    q.hza = f2(p.hza);
    q.hom = f2(p.hom);
    q.hcT2 = f2(p.hcT2);
    return q;
}

// Directions whose source lies in the same column (e_x = 0): for two nodes
// (x0, x0 + 1) with x0 even their sources are adjacent and 4-byte aligned.
__device__ __forceinline__ constexpr bool column_dir(int i) { return i == 0 || i == 2 || i == 4; }

// ---------------------------------------------------------------- storage
// Loads of the distribution buffers (stores use __stwb: explicitly global
// even where the pointer comes from shared memory, as in the batch
// kernels).  A kernel that only reads its input
// buffer takes the read-only (non-coherent) cache path.  The persistent
// batch kernel reads, in one step, what other blocks wrote in the step
// before, which the read-only path does not allow; it uses ordinary
// (coherent) loads, L2-only ones (LdCG) or L1-cached ones (LdCA), made
// consistent by the acquire fence after its grid barrier.
// The FP16 forms' read-only loads (halves, half pairs, node records) carry
// an L2 prefetch-size hint (.L2::256B): a warp's 128-byte line brings its
// neighbour into L2 with it.  Measured at 8192^2: F16S +0.7 %, F16N +0.4 %,
// the 512-case batch +0.75 % (0 turns it off; 128 measured no gain).
#ifndef CLB_LD_L2_PREFETCH
#define CLB_LD_L2_PREFETCH 256
#endif
struct LdNC {
    template <class T>
    static __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }
#if CLB_LD_L2_PREFETCH
#define CLB_STR2_(x) #x
#define CLB_STR_(x) CLB_STR2_(x)
#define CLB_L2PF_ ".L2::" CLB_STR_(CLB_LD_L2_PREFETCH) "B"
    static __device__ __forceinline__ __half ld(const __half* p) {
        unsigned short v;
        asm("ld.global.nc" CLB_L2PF_ ".b16 %0, [%1];" : "=h"(v) : "l"(p));
        return __ushort_as_half(v);
    }
    static __device__ __forceinline__ __half2 ld(const __half2* p) {
        unsigned v;
        asm("ld.global.nc" CLB_L2PF_ ".b32 %0, [%1];" : "=r"(v) : "l"(p));
        return *reinterpret_cast<const __half2*>(&v);
    }
    static __device__ __forceinline__ uint2 ld(const uint2* p) {
        uint2 v;
        asm("ld.global.nc" CLB_L2PF_ ".v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
        return v;
    }
    static __device__ __forceinline__ uint4 ld(const uint4* p) {
        uint4 v;
        asm("ld.global.nc" CLB_L2PF_ ".v4.u32 {%0, %1, %2, %3}, [%4];"
            : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
        return v;
    }
#endif
    static __device__ __forceinline__ double ld_again(const double* p) {
        double v;
        asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
        return v;
    }
};
struct LdCG {
    template <class T>
    static __device__ __forceinline__ T ld(const T* p) { return __ldcg(p); }
    static __device__ __forceinline__ double ld_again(const double* p) {
        double v;
        asm volatile("ld.global.cg.f64 %0, [%1];" : "=d"(v) : "l"(p));
        return v;
    }
};

struct LdCA {
    template <class T>
    static __device__ __forceinline__ T ld(const T* p) { return __ldca(p); }
    static __device__ __forceinline__ double ld_again(const double* p) {
        double v;
        asm volatile("ld.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
        return v;
    }
};

// A storage policy reads the streamed values of a node (pull9 / pull5),
// writes a node's post-collision values (store) and gives the per-node
// constants (coef).  L: how the distribution buffers are loaded.
template <class L>
struct StoreF64T {
    using Ld = L;
    static constexpr bool kCentred = false;   // g and T carried as they are
#ifndef CLB_F64_RELOAD
#define CLB_F64_RELOAD 1
#endif
    static constexpr bool kReload = CLB_F64_RELOAD != 0;   // interior f re-read before the update (see step_interior)
    using R = double;
    using S = double;
    static __device__ __forceinline__ void pull9(const BufT<const S>& B, const AuxT<R>&, const KParamsT<R>& K, int x,
                                                 int y, R (&f)[9]) {
        long long o[9];
        sources<long long>(K.g, x, y, o);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = L::ld(B.f + i * K.g.plane + o[i]);
    }
    static __device__ __forceinline__ void pull5(const BufT<const S>& B, const AuxT<R>&, const KParamsT<R>& K, int x,
                                                 int y, R (&g)[5]) {
        long long o[9];
        sources<long long>(K.g, x, y, o);
#pragma unroll
        for (int i = 0; i < 5; ++i) g[i] = L::ld(B.g + i * K.g.plane + o[i]);
    }
    static __device__ __forceinline__ void pull(const BufT<const S>& B, const AuxT<R>& A, const KParamsT<R>& K, int x,
                                                int y, R (&f)[9], R (&g)[5]) {
        pull9(B, A, K, x, y, f);
        pull5(B, A, K, x, y, g);
    }
    // The same nine values as pull9, loaded again (volatile: not merged
    // with the first load, so f need not stay in registers in between).
    static __device__ __forceinline__ void reload9(const BufT<const S>& B, const KParamsT<R>& K, int x, int y,
                                                   R (&f)[9]) {
        long long o[9];
        sources<long long>(K.g, x, y, o);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = L::ld_again(B.f + i * K.g.plane + o[i]);
    }
    static __device__ __forceinline__ void store(const BufT<S>& B, const KParamsT<R>& K, int x, int y,
                                                 const R (&f)[9], const R (&g)[5], R, R, R, R, R, uint32_t) {
        const long long o = (long long)y * K.g.px + x;
#pragma unroll
        for (int i = 0; i < 9; ++i) __stwb(B.f + i * K.g.plane + o, f[i]);
#pragma unroll
        for (int i = 0; i < 5; ++i) __stwb(B.g + i * K.g.plane + o, g[i]);
    }
    template <bool FORCH>
    static __device__ __forceinline__ CoefT<R> coef(const AuxT<R>& A, const KParamsT<R>& K, int x, int y) {
        return A.coef[(long long)y * K.g.nx + x];
    }
};

using StoreF64 = StoreF64T<LdNC>;

// FP32 constants of a node from its porosity and its row's a_y - g beta T0
// (Eqs. 4, 5, 23).
template <bool FORCH>
__device__ __forceinline__ CoefT<float> coef_from_phi(float p, float ip, float ayg, const KParamsT<float>& K) {
    CoefT<float> c;
    const float hp = 0.5f * p;
    c.ip = ip;
    c.hdar = hp * K.nuK;
    c.l0 = fmaf(0.5f, c.hdar, 0.5f);
    c.l0sq = c.l0 * c.l0;
    // Ergun (Eq. 5): l1 = phi F_phi / (2 sqrt K) = 0.875 / sqrt(150 K phi)
    c.aux = FORCH ? K.l1c * rsqrtf(p) : recip(c.l0 + c.l0);
    c.hgx = hp * K.p.ax;
    c.hgb = hp * K.p.gbeta;
    c.hgy = hp * ayg;
    return c;
}

// The same constants for a pair of nodes on packed FP32 (bit for bit the
// values of coef_from_phi: the same operations lane by lane).
template <bool FORCH>
__device__ __forceinline__ CoefT<f2> coef2_from_phi(f2 p, f2 ip, float ayg, const KParamsT<float>& K) {
    CoefT<f2> c;
    const f2 hp = f2(0.5) * p;
    c.ip = ip;
    c.hdar = hp * f2(K.nuK);
    c.l0 = fma(f2(0.5), c.hdar, f2(0.5));
    c.l0sq = c.l0 * c.l0;
    c.aux = FORCH ? f2(K.l1c) * f2::make(rsqrtf(p.lo()), rsqrtf(p.hi())) : recip(c.l0 + c.l0);
    c.hgx = hp * f2(K.p.ax);
    c.hgb = hp * f2(K.p.gbeta);
    c.hgy = hp * f2(ayg);
    return c;
}

template <class L>
struct StoreH16T {
    using Ld = L;
    // g is carried rest-centred (g - g_rest(T0), T - T0): the stored
    // deviations are exactly that, so no baseline is added or subtracted
    static constexpr bool kCentred = true;
    static constexpr bool kReload = false;
    using R = float;
    using S = __half;
    static __device__ __forceinline__ void pull9(const BufT<const S>& B, const AuxT<R>&, const KParamsT<R>& K, int x,
                                                 int y, R (&f)[9]) {
        int o[9];
        sources<int>(K.g, x, y, o);
        const int Q = (int)K.g.plane;
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fma(__half2float(L::ld(B.f + i * Q + o[i])), kDevInv, K.wf[i]);
    }
    static __device__ __forceinline__ void pull5(const BufT<const S>& B, const AuxT<R>&, const KParamsT<R>& K, int x,
                                                 int y, R (&g)[5]) {
        int o[9];
        sources<int>(K.g, x, y, o);
        const int Q = (int)K.g.plane;
#pragma unroll
        for (int i = 0; i < 5; ++i) g[i] = __half2float(L::ld(B.g + i * Q + o[i])) * kDevInv;
    }
    static __device__ __forceinline__ void pull(const BufT<const S>& B, const AuxT<R>& A, const KParamsT<R>& K, int x,
                                                int y, R (&f)[9], R (&g)[5]) {
        pull9(B, A, K, x, y, f);
        pull5(B, A, K, x, y, g);
    }
    static __device__ __forceinline__ void store(const BufT<S>& B, const KParamsT<R>& K, int x, int y,
                                                 const R (&f)[9], const R (&g)[5], R, R, R, R, R, uint32_t seq) {
        const int o = y * K.g.px + x, Q = (int)K.g.plane;
        const Dither d = dither_for((uint32_t)o, seq);
#pragma unroll
        for (int i = 0; i < 9; ++i) __stwb(B.f + i * Q + o, sr_half((f[i] - K.wf[i]) * kDevScale, dword(d, i)));
#pragma unroll
        for (int i = 0; i < 5; ++i) __stwb(B.g + i * Q + o, sr_half(g[i] * kDevScale, dword(d, 9 + i)));
    }
    template <bool FORCH>
    static __device__ __forceinline__ CoefT<R> coef(const AuxT<R>& A, const KParamsT<R>& K, int x, int y) {
        const float p = __ldg(A.phi + y * K.g.nx + x);
        return coef_from_phi<FORCH>(p, recip(p), A.ayg[y], K);
    }
    // per node, then packed: for this form the packed version measured 3 %
    // slower (more registers live across the pull)
    template <bool FORCH>
    static __device__ __forceinline__ CoefT<f2> coef2(const AuxT<R>& A, const KParamsT<R>& K, int x0, int y) {
        const CoefT<float> a = coef<FORCH>(A, K, x0, y), b = coef<FORCH>(A, K, x0 + 1, y);
        CoefT<f2> c;
        c.ip = f2::make(a.ip, b.ip);
        c.l0 = f2::make(a.l0, b.l0);
        c.l0sq = f2::make(a.l0sq, b.l0sq);
        c.aux = f2::make(a.aux, b.aux);
        c.hdar = f2::make(a.hdar, b.hdar);
        c.hgx = f2::make(a.hgx, b.hgx);
        c.hgb = f2::make(a.hgb, b.hgb);
        c.hgy = f2::make(a.hgy, b.hgy);
        return c;
    }
    // Two interior nodes (x0, x0 + 1), x0 even, neither at the periodic x
    // seam: node x0 + 1 pulls from the offsets of node x0 plus one.
    static __device__ __forceinline__ void pull2(const BufT<const S>& B, const AuxT<R>&, const KParamsT<R>& K, int x0,
                                                 int y, f2 (&f)[9], f2 (&g)[5]) {
        int o[9];
        sources<int>(K.g, x0, y, o);
        const int Q = (int)K.g.plane;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const __half* p = B.f + i * Q + o[i];
            float2 v;
            if (column_dir(i)) v = __half22float2(L::ld(reinterpret_cast<const __half2*>(p)));
            else v = make_float2(__half2float(L::ld(p)), __half2float(L::ld(p + 1)));
            f[i] = fma(f2::make(v.x, v.y), f2(kDevInv), f2(K.wf[i]));
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const __half* p = B.g + i * Q + o[i];
            float2 v;
            if (column_dir(i)) v = __half22float2(L::ld(reinterpret_cast<const __half2*>(p)));
            else v = make_float2(__half2float(L::ld(p)), __half2float(L::ld(p + 1)));
            g[i] = f2::make(v.x, v.y) * f2(kDevInv);
        }
    }
    static __device__ __forceinline__ void store2(const BufT<S>& B, const KParamsT<R>& K, int x0, int y,
                                                  const f2 (&f)[9], const f2 (&g)[5], f2, f2, f2, f2, f2,
                                                  uint32_t seq) {
        const int o = y * K.g.px + x0, Q = (int)K.g.plane;
        const Dither rw = dither_for((uint32_t)o, seq);   // one word per stored pair
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const f2 d = fma(f[i], f2(kDevScale), f2(-K.wfs[i]));   // (f - w_i rho_0) 2^12
            __stwb(reinterpret_cast<__half2*>(B.f + i * Q + o), sr_half2(d.lo(), d.hi(), dword(rw, i)));
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const f2 d = g[i] * f2(kDevScale);
            __stwb(reinterpret_cast<__half2*>(B.g + i * Q + o), sr_half2(d.lo(), d.hi(), dword(rw, 9 + i)));
        }
    }
};

using StoreH16 = StoreH16T<LdNC>;

// Baseline (rho, u, T - T0, 1/phi) of the node whose record sits at plane offset o.
struct Base {
    float rho, X, Y, Tt, ip;
};

template <class L>
__device__ __forceinline__ Base load_base(const BufT<const __half>& B, const AuxT<float>& A,
                                          const KParamsT<float>& K, int o) {
    const uint2 r = L::ld(B.rec + o);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
    Base s;
    s.rho = 1.0f + a.x;
    s.X = a.y;
    s.Y = b.x;
    s.Tt = b.y;
    s.ip = __ldg(A.ip + o);
    return s;
}

// One component of the porous equilibrium f^eq = M^-1 m^eq (Eq. 19), written
// out per direction (the value a puller needs from each source).  With
// A = rho / phi, S = X^2 + Y^2 and, for direction e_i, the signed velocity
// components a = e_ix X, b = e_iy Y:
//   f0       = (4/9) rho + A (ip X^2 Y^2 - (2/3) S)
//   f1..4    = rho (1/9 + d/3) - (A/2) (o^2 (1/3 + d + ip d^2) - (2/3) d^2),
//              d = the signed component along e_i, o the other one
//   f5..8    = rho (1/36 + s/12) + (A/4) (S/3 + ab (1 + s) + ip (XY)^2),  s = a + b
// (the cubic and quartic terms of Eq. 19 grouped so that the direction's
// signs only ever select constants or an addition against a subtraction:
// the packed type has no free negation).
template <int I, typename R>
__device__ __forceinline__ R feq_comp(R rho, R X, R Y, R ip) {
    if (I == 0) {
        const R X2 = X * X, Y2 = Y * Y;
        return fma(rho * ip, fma(ip * X2, Y2, R(-2.0 / 3.0) * (X2 + Y2)), rho * R(4.0 / 9.0));
    } else if (I <= 4) {
        constexpr bool pos = I <= 2;                                   // e_i along +x or +y
        const R u = (I == 1 || I == 3) ? X : Y, o = (I == 1 || I == 3) ? Y : X;
        const R d2 = u * u;
        const R w = fma(ip, d2, pos ? u + R(1.0 / 3.0) : R(1.0 / 3.0) - u);   // 1/3 + d + ip d^2
        const R tn = fma(o * o, w, R(-2.0 / 3.0) * d2);
        return fma(rho * (R(-0.5) * ip), tn, rho * fma(u, R(pos ? 1.0 / 3.0 : -1.0 / 3.0), R(1.0 / 9.0)));
    } else {
        // s holds a + b, except for I = 7 (a + b = -(X + Y)), where it holds X + Y
        const R XY = X * Y;
        const R s = I == 5 || I == 7 ? X + Y : (I == 6 ? Y - X : X - Y);
        // ab (1 + a + b) = XY c:  c = 1 + s (I = 5), 1 - s (I = 7), -1 - s (I = 6, 8)
        const R c = I == 5 ? s + R(1.0) : (I == 7 ? R(1.0) - s : R(-1.0) - s);
        const R t = fma(R(1.0 / 3.0), fma(X, X, Y * Y), fma(XY, c, (ip * XY) * XY));
        return fma(rho * (R(0.25) * ip), t, rho * fma(s, R(I == 7 ? -1.0 / 12.0 : 1.0 / 12.0), R(1.0 / 36.0)));
    }
}

template <int I, class L>
__device__ __forceinline__ void pull_one(const BufT<const __half>& B, const AuxT<float>& A, const KParamsT<float>& K,
                                         const int (&o)[9], float (&f)[9], float (&g)[5], bool want_f, bool want_g) {
    const Base s = load_base<L>(B, A, K, o[I]);
    const int Q = (int)K.g.plane;
    if (want_f) f[I] = fma(__half2float(L::ld(B.f + I * Q + o[I])), kDevInv, feq_comp<I>(s.rho, s.X, s.Y, s.ip));
    if (I < 5 && want_g)
        g[I < 5 ? I : 0] = fma(__half2float(L::ld(B.g + (I < 5 ? I : 0) * Q + o[I])), kDevInv,
                               geqc_comp<(I < 5 ? I : 0)>(s.Tt, s.X, s.Y, K.p.sigma, K.p.cT2, K.T0));
}

template <class L>
struct StoreH16NT {
    using Ld = L;
    static constexpr bool kCentred = true;    // g - g_rest(T0) and T - T0 (see geqc_comp)
    static constexpr bool kReload = false;
    using R = float;
    using S = __half;
    static __device__ __forceinline__ void pull_all(const BufT<const S>& B, const AuxT<R>& A, const KParamsT<R>& K,
                                                    int x, int y, R (&f)[9], R (&g)[5], bool wf, bool wg) {
        int o[9];
        sources<int>(K.g, x, y, o);
        pull_one<0, L>(B, A, K, o, f, g, wf, wg);
        pull_one<1, L>(B, A, K, o, f, g, wf, wg);
        pull_one<2, L>(B, A, K, o, f, g, wf, wg);
        pull_one<3, L>(B, A, K, o, f, g, wf, wg);
        pull_one<4, L>(B, A, K, o, f, g, wf, wg);
        pull_one<5, L>(B, A, K, o, f, g, wf, wg);
        pull_one<6, L>(B, A, K, o, f, g, wf, wg);
        pull_one<7, L>(B, A, K, o, f, g, wf, wg);
        pull_one<8, L>(B, A, K, o, f, g, wf, wg);
    }
    static __device__ __forceinline__ void pull9(const BufT<const S>& B, const AuxT<R>& A, const KParamsT<R>& K, int x,
                                                 int y, R (&f)[9]) {
        R g[5];
        pull_all(B, A, K, x, y, f, g, true, false);
    }
    static __device__ __forceinline__ void pull5(const BufT<const S>& B, const AuxT<R>& A, const KParamsT<R>& K, int x,
                                                 int y, R (&g)[5]) {
        R f[9];
        pull_all(B, A, K, x, y, f, g, false, true);
    }
    static __device__ __forceinline__ void pull(const BufT<const S>& B, const AuxT<R>& A, const KParamsT<R>& K, int x,
                                                int y, R (&f)[9], R (&g)[5]) {
        pull_all(B, A, K, x, y, f, g, true, true);
    }
    // The record is rounded first and the baseline rebuilt from the rounded
    // halves, exactly as a reader will rebuild it.
    static __device__ __forceinline__ void store(const BufT<S>& B, const KParamsT<R>& K, int x, int y,
                                                 const R (&f)[9], const R (&g)[5], R rho, R X, R Y, R T, R ip,
                                                 uint32_t seq) {
        const int o = y * K.g.px + x, Q = (int)K.g.plane;
        const __half2 a = __floats2half2_rn(rho - 1.0f, X);
        const __half2 b = __floats2half2_rn(Y, T);              // T: T - T0 in this form
        uint2 r;
        r.x = *reinterpret_cast<const unsigned int*>(&a);
        r.y = *reinterpret_cast<const unsigned int*>(&b);
        __stwb(B.rec + o, r);
        // same per-direction formulas, on the same rounded record, as pull_one
        const float2 fa = __half22float2(a), fb = __half22float2(b);
        const float br = 1.0f + fa.x, bX = fa.y, bY = fb.x, bT = fb.y;
        const float fe[9] = {feq_comp<0>(br, bX, bY, ip), feq_comp<1>(br, bX, bY, ip), feq_comp<2>(br, bX, bY, ip),
                             feq_comp<3>(br, bX, bY, ip), feq_comp<4>(br, bX, bY, ip), feq_comp<5>(br, bX, bY, ip),
                             feq_comp<6>(br, bX, bY, ip), feq_comp<7>(br, bX, bY, ip), feq_comp<8>(br, bX, bY, ip)};
        const float s = K.p.sigma, c = K.p.cT2;
        const float t0 = K.T0;
        const float ge[5] = {geqc_comp<0>(bT, bX, bY, s, c, t0), geqc_comp<1>(bT, bX, bY, s, c, t0),
                             geqc_comp<2>(bT, bX, bY, s, c, t0), geqc_comp<3>(bT, bX, bY, s, c, t0),
                             geqc_comp<4>(bT, bX, bY, s, c, t0)};
        const Dither d = dither_for((uint32_t)o, seq);
#pragma unroll
        for (int i = 0; i < 9; ++i) __stwb(B.f + i * Q + o, sr_half((f[i] - fe[i]) * kDevScale, dword(d, i)));
#pragma unroll
        for (int i = 0; i < 5; ++i) __stwb(B.g + i * Q + o, sr_half((g[i] - ge[i]) * kDevScale, dword(d, 9 + i)));
    }
    template <bool FORCH>
    static __device__ __forceinline__ CoefT<R> coef(const AuxT<R>& A, const KParamsT<R>& K, int x, int y) {
        const float ip = __ldg(A.ip + y * K.g.px + x);
        return coef_from_phi<FORCH>(recip(ip), ip, A.ayg[y], K);
    }
    template <bool FORCH>
    static __device__ __forceinline__ CoefT<f2> coef2(const AuxT<R>& A, const KParamsT<R>& K, int x0, int y) {
        const float2 q = __ldg(reinterpret_cast<const float2*>(A.ip + y * K.g.px + x0));   // x0 and px even
        const f2 ip = f2::make(q.x, q.y);
        return coef2_from_phi<FORCH>(recip(ip), ip, A.ayg[y], K);
    }
    // Two interior nodes (x0, x0 + 1), x0 even, neither at the periodic x
    // seam (node x0 + 1 pulls from node x0's offsets plus one).
    template <int I>
    static __device__ __forceinline__ void pull2_one(const BufT<const S>& B, const AuxT<R>& A, const KParamsT<R>& K,
                                                     const int (&o0)[9], f2 (&f)[9], f2 (&g)[5]) {
        const int Q = (int)K.g.plane;
        uint2 r0, r1;
        float2 ip, df, dg = make_float2(0.0f, 0.0f);
        if (column_dir(I)) {
            const uint4 r = L::ld(reinterpret_cast<const uint4*>(B.rec + o0[I]));
            r0 = make_uint2(r.x, r.y);
            r1 = make_uint2(r.z, r.w);
            ip = __ldg(reinterpret_cast<const float2*>(A.ip + o0[I]));
            df = __half22float2(L::ld(reinterpret_cast<const __half2*>(B.f + I * Q + o0[I])));
            if (I < 5) dg = __half22float2(L::ld(reinterpret_cast<const __half2*>(B.g + (I < 5 ? I : 0) * Q + o0[I])));
        } else {
            r0 = L::ld(B.rec + o0[I]);
            r1 = L::ld(B.rec + o0[I] + 1);
            ip = make_float2(__ldg(A.ip + o0[I]), __ldg(A.ip + o0[I] + 1));
            df = make_float2(__half2float(L::ld(B.f + I * Q + o0[I])), __half2float(L::ld(B.f + I * Q + o0[I] + 1)));
            if (I < 5)
                dg = make_float2(__half2float(L::ld(B.g + (I < 5 ? I : 0) * Q + o0[I])),
                                 __half2float(L::ld(B.g + (I < 5 ? I : 0) * Q + o0[I] + 1)));
        }
        combine2<I>(r0, r1, ip, df, dg, K, f, g);
    }
    // Streamed values of direction I for the pair from the sources' records
    // r0, r1, their 1/phi and the stored deviations df (and dg, I < 5).
    template <int I>
    static __device__ __forceinline__ void combine2(uint2 r0, uint2 r1, float2 ip, float2 df, float2 dg,
                                                    const KParamsT<R>& K, f2 (&f)[9], f2 (&g)[5]) {
        const float2 a0 = __half22float2(*reinterpret_cast<const __half2*>(&r0.x));
        const float2 b0 = __half22float2(*reinterpret_cast<const __half2*>(&r0.y));
        const float2 a1 = __half22float2(*reinterpret_cast<const __half2*>(&r1.x));
        const float2 b1 = __half22float2(*reinterpret_cast<const __half2*>(&r1.y));
        const f2 rho = f2(1.0) + f2::make(a0.x, a1.x), X = f2::make(a0.y, a1.y), Y = f2::make(b0.x, b1.x);
        const f2 ipp = f2::make(ip.x, ip.y);
        f[I] = fma(f2::make(df.x, df.y), f2(kDevInv), feq_comp<I>(rho, X, Y, ipp));
        if (I < 5) {
            const f2 Tt = f2::make(b0.y, b1.y);
            g[I < 5 ? I : 0] = fma(f2::make(dg.x, dg.y), f2(kDevInv),
                                   geqc_comp<(I < 5 ? I : 0)>(Tt, X, Y, f2(K.p.sigma), f2(K.p.cT2), f2(K.T0)));
        }
    }
    static __device__ __forceinline__ void pull2(const BufT<const S>& B, const AuxT<R>& A, const KParamsT<R>& K, int x0,
                                                 int y, f2 (&f)[9], f2 (&g)[5]) {
        int o0[9];                                   // node x0 + 1: the same offsets plus one
        sources<int>(K.g, x0, y, o0);
        pull2_one<0>(B, A, K, o0, f, g);
        pull2_one<1>(B, A, K, o0, f, g);
        pull2_one<2>(B, A, K, o0, f, g);
        pull2_one<3>(B, A, K, o0, f, g);
        pull2_one<4>(B, A, K, o0, f, g);
        pull2_one<5>(B, A, K, o0, f, g);
        pull2_one<6>(B, A, K, o0, f, g);
        pull2_one<7>(B, A, K, o0, f, g);
        pull2_one<8>(B, A, K, o0, f, g);
    }
    static __device__ __forceinline__ void store2(const BufT<S>& B, const KParamsT<R>& K, int x0, int y,
                                                  const f2 (&f)[9], const f2 (&g)[5], f2 rho, f2 X, f2 Y, f2 T, f2 ip,
                                                  uint32_t seq) {
        const int o = y * K.g.px + x0, Q = (int)K.g.plane;
        // T: T - T0 in this form
        const __half2 a0 = __floats2half2_rn(rho.lo() - 1.0f, X.lo()), b0 = __floats2half2_rn(Y.lo(), T.lo());
        const __half2 a1 = __floats2half2_rn(rho.hi() - 1.0f, X.hi()), b1 = __floats2half2_rn(Y.hi(), T.hi());
        uint4 r;
        r.x = *reinterpret_cast<const unsigned int*>(&a0);
        r.y = *reinterpret_cast<const unsigned int*>(&b0);
        r.z = *reinterpret_cast<const unsigned int*>(&a1);
        r.w = *reinterpret_cast<const unsigned int*>(&b1);
        __stwb(reinterpret_cast<uint4*>(B.rec + o), r);
        const float2 fa0 = __half22float2(a0), fb0 = __half22float2(b0);
        const float2 fa1 = __half22float2(a1), fb1 = __half22float2(b1);
        const f2 br = f2(1.0) + f2::make(fa0.x, fa1.x), bX = f2::make(fa0.y, fa1.y), bY = f2::make(fb0.x, fb1.x);
        const f2 bT = f2::make(fb0.y, fb1.y), t0 = f2(K.T0);
        const f2 fe[9] = {feq_comp<0>(br, bX, bY, ip), feq_comp<1>(br, bX, bY, ip), feq_comp<2>(br, bX, bY, ip),
                          feq_comp<3>(br, bX, bY, ip), feq_comp<4>(br, bX, bY, ip), feq_comp<5>(br, bX, bY, ip),
                          feq_comp<6>(br, bX, bY, ip), feq_comp<7>(br, bX, bY, ip), feq_comp<8>(br, bX, bY, ip)};
        const f2 s = f2(K.p.sigma), c = f2(K.p.cT2);
        const f2 ge[5] = {geqc_comp<0>(bT, bX, bY, s, c, t0), geqc_comp<1>(bT, bX, bY, s, c, t0),
                          geqc_comp<2>(bT, bX, bY, s, c, t0), geqc_comp<3>(bT, bX, bY, s, c, t0),
                          geqc_comp<4>(bT, bX, bY, s, c, t0)};
        const Dither rw = dither_for((uint32_t)o, seq);   // one word per stored pair
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const f2 d = (f[i] - fe[i]) * f2(kDevScale);
            __stwb(reinterpret_cast<__half2*>(B.f + i * Q + o), sr_half2(d.lo(), d.hi(), dword(rw, i)));
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const f2 d = (g[i] - ge[i]) * f2(kDevScale);
            __stwb(reinterpret_cast<__half2*>(B.g + i * Q + o), sr_half2(d.lo(), d.hi(), dword(rw, 9 + i)));
        }
    }
};

using StoreH16N = StoreH16NT<LdNC>;

// Inward normal of a wall node and the sides that set its velocity and
// temperature.  Returns false for an interior node.
struct WallInfo {
    int dx, dy, su, st;
};

template <typename R>
__device__ __forceinline__ bool wall_info(const Geo& G, const BndT<R>& B, int x, int y, WallInfo& w) {
    int vs = -1, hs = -1;
    w.dx = 0;
    w.dy = 0;
    if (G.wall_x) {
        if (x == 0) { w.dx = 1; vs = 0; }
        else if (x == G.nx - 1) { w.dx = -1; vs = 1; }
    }
    if (G.wall_y) {
        if (y == 0) { w.dy = 1; hs = 2; }
        else if (y == G.ny - 1) { w.dy = -1; hs = 3; }
    }
    if (vs < 0 && hs < 0) return false;
    w.su = vs >= 0 ? vs : hs;
    w.st = (vs >= 0 && B.iso[vs]) ? vs : ((hs >= 0 && B.iso[hs]) ? hs : -1);
    return true;
}

// Pre-collision state of a wall node by non-equilibrium extrapolation from
// its inward neighbour s = (x + dx, y + dy), pulled here from the same
// post-collision buffer as every other node:
//   f(b) = f^eq(rho_s, u_w; phi_b) + f(s) - f^eq(rho_s, u_s; phi_s)
//   g(b) = g^eq(T_b, u_w) + g(s) - g^eq(T_s, u_s)
// T_b = T_w (isothermal) or (4 T_s - T_ss) / 3 (adiabatic).
template <class P, bool FORCH>
__device__ __forceinline__ void wall_state(const BufT<const typename P::S>& Bin, const AuxT<typename P::R>& A,
                                           const KParamsT<typename P::R>& K, int x, int y, const WallInfo& w,
                                           const CoefT<typename P::R>& cb, typename P::R (&f)[9],
                                           typename P::R (&g)[5], typename P::R& rho, typename P::R& X,
                                           typename P::R& Y, typename P::R& T, typename P::R& Tt,
                                           typename P::R& n0) {
    using R = typename P::R;
    // temperatures below are in the form's representation (T - T0 in the
    // rest-centred form, T otherwise); T itself is returned for the force
    const int sx = x + w.dx, sy = y + w.dy;
    R fs[9], gs[5];
    P::pull(Bin, A, K, sx, sy, fs, gs);
    const Mom9T<R> ks = moments9(fs);
    const R Tst = sum5(gs) * K.p.inv_sigma;
    R Ts = Tst;
    if constexpr (P::kCentred) Ts = R(K.T0) + Tst;
    const CoefT<R> cs = P::template coef<FORCH>(A, K, sx, sy);
    R Xs, Ys, hFxs, hFys;
    macro_velocity<R, FORCH>(ks.rho, ks.jx, ks.jy, Ts, cs, Xs, Ys, hFxs, hFys);
    R Tbt;
    if (w.st >= 0) {
        Tbt = K.b.Tw[w.st];
        if constexpr (P::kCentred) Tbt = Tbt - R(K.T0);
    } else {
        R gss[5];
        P::pull5(Bin, A, K, x + 2 * w.dx, y + 2 * w.dy, gss);
        const R Tsst = sum5(gss) * K.p.inv_sigma;
        Tbt = (R(4) * Tst - Tsst) * R(1.0 / 3.0);
    }
    const R uw = K.b.uw[w.su], vw = K.b.vw[w.su];
    R fb[9], fe[9];
    feq9(ks.rho, uw, vw, cb.ip, fb);
    feq9(ks.rho, Xs, Ys, cs.ip, fe);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = fb[i] + (fs[i] - fe[i]);
    R gb[5], ge[5];
    if constexpr (P::kCentred) {
        geq5c(Tbt, uw, vw, K.p.sigma, K.p.cT2, R(K.T0), gb);
        geq5c(Tst, Xs, Ys, K.p.sigma, K.p.cT2, R(K.T0), ge);
    } else {
        geq5(Tbt, uw, vw, K.p.sigma, K.p.cT2, gb);
        geq5(Tst, Xs, Ys, K.p.sigma, K.p.cT2, ge);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) g[i] = gb[i] + (gs[i] - ge[i]);
    rho = ks.rho;
    X = uw;
    Y = vw;
    Tt = Tbt;
    T = Tbt;
    if constexpr (P::kCentred) T = R(K.T0) + Tbt;
    n0 = sum5(g);
}

// Macroscopic state of any node at the current time level (pre-collision
// values in f, g; wall nodes rebuilt by non-equilibrium extrapolation).  T
// is the temperature, Tt and n0 = sigma Tt the form's representation of it
// (equal to T and sum g unless the form is rest-centred).
template <class P, bool FORCH>
__device__ __forceinline__ void node_state(const BufT<const typename P::S>& Bin, const AuxT<typename P::R>& A,
                                           const KParamsT<typename P::R>& K, int x, int y,
                                           const CoefT<typename P::R>& c, typename P::R (&f)[9],
                                           typename P::R (&g)[5], Mom9T<typename P::R>& k, typename P::R& rho,
                                           typename P::R& X, typename P::R& Y, typename P::R& T,
                                           typename P::R& Tt, typename P::R& hFx, typename P::R& hFy,
                                           typename P::R& n0) {
    using R = typename P::R;
    WallInfo w;
    if (!wall_info(K.g, K.b, x, y, w)) {
        P::pull(Bin, A, K, x, y, f, g);
        k = moments9(f);
        n0 = sum5(g);
        Tt = n0 * K.p.inv_sigma;
        T = Tt;
        if constexpr (P::kCentred) T = R(K.T0) + Tt;
        rho = k.rho;
        macro_velocity<R, FORCH>(rho, k.jx, k.jy, T, c, X, Y, hFx, hFy);
    } else {
        wall_state<P, FORCH>(Bin, A, K, x, y, w, c, f, g, rho, X, Y, T, Tt, n0);
        k = moments9(f);
        force_at<R, FORCH>(X, Y, T, c, hFx, hFy);
    }
}

// ---------------------------------------------------------------- kernels
// Step counter of the input buffer (FP16 forms; 0 without one); the thread
// of node (0, 0) writes the next value into the output buffer, which no
// thread of this launch reads.
template <class L, typename S>
__device__ __forceinline__ uint32_t step_seq(const BufT<S>& in, const BufT<S>& out, int x, int y) {
    if (!in.seq) return 0U;
    const uint32_t seq = L::ld(in.seq);
    if (x == 0 && y == 0) __stwb(out.seq, seq + 1U);
    return seq;
}

// One node's complete step: pull (or wall rebuild), macros, both collisions, store.
// Interior nodes of a form with P::kReload drop f after taking its moments
// and read it again from the input buffer (an L1/L2 hit) just before the
// update f* = f + M^-1 r: nine loads instead of eighteen registers held
// through the collision, which buys occupancy for the FP64-bound step.
template <class P, bool SHIFT, bool FORCH>
__device__ __forceinline__ void step_interior(const BufT<typename P::S>& in, const BufT<typename P::S>& out,
                                              const AuxT<typename P::R>& A, const KParamsT<typename P::R>& K,
                                              int x, int y) {
    using R = typename P::R;
    const CoefT<R> c = P::template coef<FORCH>(A, K, x, y);
    const uint32_t seq = step_seq<typename P::Ld>(in, out, x, y);
    R f[9], g[5];
    P::pull(as_const(in), A, K, x, y, f, g);
    const Mom9T<R> k = moments9(f);
    const R n0 = sum5(g);
    const R Tt = n0 * K.p.inv_sigma;
    R T = Tt;
    if constexpr (P::kCentred) T = R(K.T0) + Tt;
    R X, Y, hFx, hFy;
    macro_velocity<R, FORCH>(k.rho, k.jx, k.jy, T, c, X, Y, hFx, hFy);
    const Incr9T<R> r = collide9_incr<R, SHIFT>(k, k.rho, X, Y, hFx, hFy, c.ip, K.p);
    if constexpr (P::kCentred) collide5_centred<R, SHIFT>(g, n0, Tt, X, Y, R(K.T0), K.p);
    else collide5<R, SHIFT>(g, n0, T, X, Y, K.p);
    if constexpr (P::kReload) P::reload9(as_const(in), K, x, y, f);
    apply9(f, r);
    P::store(out, K, x, y, f, g, k.rho, X, Y, Tt, c.ip, seq);
}

template <class P, bool SHIFT, bool FORCH>
__device__ __forceinline__ void step_wall(const BufT<typename P::S>& in, const BufT<typename P::S>& out,
                                          const AuxT<typename P::R>& A, const KParamsT<typename P::R>& K, int x,
                                          int y, const WallInfo& w) {
    using R = typename P::R;
    const CoefT<R> c = P::template coef<FORCH>(A, K, x, y);
    const uint32_t seq = step_seq<typename P::Ld>(in, out, x, y);
    R f[9], g[5];
    R rho, X, Y, T, Tt, hFx, hFy, n0;
    wall_state<P, FORCH>(as_const(in), A, K, x, y, w, c, f, g, rho, X, Y, T, Tt, n0);
    const Mom9T<R> k = moments9(f);
    force_at<R, FORCH>(X, Y, T, c, hFx, hFy);
    collide9<R, SHIFT>(f, k, rho, X, Y, hFx, hFy, c.ip, K.p);
    if constexpr (P::kCentred) collide5_centred<R, SHIFT>(g, n0, Tt, X, Y, R(K.T0), K.p);
    else collide5<R, SHIFT>(g, n0, T, X, Y, K.p);
    P::store(out, K, x, y, f, g, rho, X, Y, Tt, c.ip, seq);
}

template <class P, bool SHIFT, bool FORCH>
__device__ __forceinline__ void step_node(const BufT<typename P::S>& in, const BufT<typename P::S>& out,
                                          const AuxT<typename P::R>& A, const KParamsT<typename P::R>& K, int x,
                                          int y) {
    WallInfo w;
    if (!wall_info(K.g, K.b, x, y, w)) step_interior<P, SHIFT, FORCH>(in, out, A, K, x, y);
    else step_wall<P, SHIFT, FORCH>(in, out, A, K, x, y, w);
}

// Number of wall nodes, and the i-th of them: the S and N rows first (if
// walled), then the W and E columns without the corners already counted.
__host__ __device__ inline long long wall_count(const Geo& G) {
    long long n = 0;
    if (G.wall_y) n += 2LL * G.nx;
    if (G.wall_x) n += 2LL * (G.wall_y ? G.ny - 2 : G.ny);
    return n;
}

__device__ __forceinline__ void wall_node(const Geo& G, int i, int& x, int& y) {
    if (G.wall_y) {
        if (i < G.nx) { x = i; y = 0; return; }
        if (i < 2 * G.nx) { x = i - G.nx; y = G.ny - 1; return; }
        i -= 2 * G.nx;
        const int h = G.ny - 2;
        x = i < h ? 0 : G.nx - 1;
        y = 1 + (i < h ? i : i - h);
        return;
    }
    x = i < G.ny ? 0 : G.nx - 1;
    y = i < G.ny ? i : i - G.ny;
}

// FP64 step launch shape: threads per block (x extent CLB_F64_BX) and the
// resident blocks per SM the register allocation is capped for.  Measured
// at 4096^2 (GB300): 128 threads, 5 blocks (<= 96 registers, 20 warps/SM)
// 2.98 GLUPS; 256 x 2 blocks 2.97; 6 or 7 blocks of 128 spill and run at
// 2.88 / 2.96.
#ifndef CLB_F64_THREADS
#define CLB_F64_THREADS 128
#endif
#ifndef CLB_F64_MINB
#define CLB_F64_MINB 5
#endif
#ifndef CLB_F64_BX
#define CLB_F64_BX 64
#endif

// One launch, two kinds of blocks, so that no warp mixes the interior and
// the wall path: blocks [0, n_tiles) cover the grid in tiles_x x ... tiles
// of blockDim nodes and skip wall nodes; the blocks after them take the
// wall nodes, one per thread, in wall_node order.
template <class P, bool SHIFT, bool FORCH>
__global__ void __launch_bounds__(CLB_F64_THREADS, CLB_F64_MINB)
    k_step(const BufT<typename P::S> in, const BufT<typename P::S> out, const AuxT<typename P::R> A,
           const KParamsT<typename P::R> K, int tiles_x, int n_tiles) {
    const int b = blockIdx.x;
    if (b < n_tiles) {
        const int x = (b % tiles_x) * blockDim.x + threadIdx.x;
        const int y = (b / tiles_x) * blockDim.y + threadIdx.y;
        if (x >= K.g.nx || y >= K.g.ny) return;
        if ((K.g.wall_x && (x == 0 || x == K.g.nx - 1)) || (K.g.wall_y && (y == 0 || y == K.g.ny - 1))) return;
        step_interior<P, SHIFT, FORCH>(in, out, A, K, x, y);
    } else {
        const long long i = (long long)(b - n_tiles) * (blockDim.x * blockDim.y) + threadIdx.y * blockDim.x +
                            threadIdx.x;
        if (i >= wall_count(K.g)) return;
        int x, y;
        wall_node(K.g, (int)i, x, y);
        WallInfo w;
        wall_info(K.g, K.b, x, y, w);
        step_wall<P, SHIFT, FORCH>(in, out, A, K, x, y, w);
    }
}

// FP16 forms, two nodes (x0, x0 + 1) per thread: interior pairs run the
// collision on packed FP32 pairs.  A pair that touches a wall, the first
// and the last pair of a row (at a periodic x seam node x0 + 1 would not
// pull from node x0's offsets plus one) and the odd last column fall back
// to the per-node path.
// Macroscopic state, both collisions and the store of an interior pair
// whose streamed values f, g (pre-collision, the form's representation)
// have been pulled; c: the pair's constants, P2: the model parameters on
// pairs, seq: the input buffer's step counter.
template <class P, bool SHIFT, bool FORCH>
__device__ __forceinline__ void collide_store_pair(f2 (&f)[9], f2 (&g)[5], const CoefT<f2>& c, const PhysT<f2>& P2,
                                                   const BufT<typename P::S>& out, const KParamsT<float>& K, int x0,
                                                   int y, uint32_t seq) {
    const Mom9T<f2> k = moments9(f);
    const f2 n0 = sum5(g);
    const f2 Tt = n0 * P2.inv_sigma;          // the form's representation of T
    f2 T = Tt;
    if constexpr (P::kCentred) T = f2(K.T0) + Tt;
    f2 X, Y, hFx, hFy;
    macro_velocity<f2, FORCH>(k.rho, k.jx, k.jy, T, c, X, Y, hFx, hFy);
    collide9<f2, SHIFT>(f, k, k.rho, X, Y, hFx, hFy, c.ip, P2);
    if constexpr (P::kCentred) collide5_centred<f2, SHIFT>(g, n0, Tt, X, Y, f2(K.T0), P2);
    else collide5<f2, SHIFT>(g, n0, T, X, Y, P2);
    P::store2(out, K, x0, y, f, g, k.rho, X, Y, Tt, c.ip, seq);
}

template <class P, bool SHIFT, bool FORCH>
__device__ __forceinline__ void step_pair_interior(const BufT<typename P::S>& in, const BufT<typename P::S>& out,
                                                   const AuxT<float>& A, const KParamsT<float>& K, int x0, int y) {
    const PhysT<f2> P2 = splat(K.p);
    const CoefT<f2> c = P::template coef2<FORCH>(A, K, x0, y);
    f2 f[9], g[5];
    P::pull2(as_const(in), A, K, x0, y, f, g);
    collide_store_pair<P, SHIFT, FORCH>(f, g, c, P2, out, K, x0, y, step_seq<typename P::Ld>(in, out, x0, y));
}

// True if the pair (x0, x0 + 1) takes the packed path.
__device__ __forceinline__ bool interior_pair(const Geo& G, int x0, int y) {
    return x0 > 0 && x0 + 2 < G.nx && !(G.wall_y && (y == 0 || y == G.ny - 1));
}

template <class P, bool SHIFT, bool FORCH>
__device__ __forceinline__ void step_pair(const BufT<typename P::S>& in, const BufT<typename P::S>& out,
                                          const AuxT<float>& A, const KParamsT<float>& K, int x0, int y) {
    if (interior_pair(K.g, x0, y)) {
        step_pair_interior<P, SHIFT, FORCH>(in, out, A, K, x0, y);
    } else {
        step_node<P, SHIFT, FORCH>(in, out, A, K, x0, y);
        if (x0 + 1 < K.g.nx) step_node<P, SHIFT, FORCH>(in, out, A, K, x0 + 1, y);
    }
}

// Nodes that the per-node path takes in k_step2 ("edge" nodes): all nodes
// of walled S/N rows, and in every other row the nodes of its first and its
// last pair (all nodes of a row with fewer than three pairs).  Count and
// the i-th one.
#ifndef CLB_EDGE_BY_COLUMN
#define CLB_EDGE_BY_COLUMN 1
#endif
__host__ __device__ inline int edge_per_row(int nx) {
    const int np = (nx + 1) / 2;
    if (np < 3) return nx;
    const int xl = 2 * (np - 1);
    return 2 + (nx - xl);   // {0, 1} and {xl, xl + 1} within the row
}

__host__ __device__ inline long long edge_count(const Geo& G) {
    const int rows = G.wall_y ? G.ny - 2 : G.ny;
    return (G.wall_y ? 2LL * G.nx : 0LL) + (long long)rows * edge_per_row(G.nx);
}

__host__ __device__ __forceinline__ void edge_node(const Geo& G, long long i, int& x, int& y) {
    if (G.wall_y) {
        if (i < G.nx) { x = (int)i; y = 0; return; }
        if (i < 2LL * G.nx) { x = (int)(i - G.nx); y = G.ny - 1; return; }
        i -= 2LL * G.nx;
    }
#if CLB_EDGE_BY_COLUMN
    // column by column (all rows of one edge column, then the next): a warp's
    // nodes are then all walls or all fluid and take one branch of step_node
    const int rows = G.wall_y ? G.ny - 2 : G.ny;
    const int k = (int)(i / rows), r = (int)(i - (long long)k * rows);
#else
    const int ne = edge_per_row(G.nx);
    const int r = (int)(i / ne), k = (int)(i - (long long)r * ne);
#endif
    y = r + (G.wall_y ? 1 : 0);
    const int np = (G.nx + 1) / 2;
    x = (np < 3 || k < 2) ? k : 2 * (np - 1) + (k - 2);
}

// One launch, two kinds of blocks (no warp mixes the packed and the
// per-node path): blocks [0, n_tiles) cover all pairs of the grid in
// tiles_x x ... tiles of blockDim pairs, aligned at x = 0 so that a warp's
// 64 nodes are one 128-byte line of every FP16 plane, and skip the pairs
// that are not interior; the blocks after them take the edge nodes, one per
// thread, with 128-thread blocks.
// Resident 128-thread blocks per SM the registers of k_step2 are capped
// for, per form (measured at 8192^2 with 64 x 2-thread blocks): the
// rest-shifted form runs 7 (72 registers, 48 bytes of spills, 28 warps:
// 78.0 GLUPS against 75.2 with 6 and 73.3 with 8); the equilibrium-shifted
// form spills below 96 registers (6 blocks: 38.1 GLUPS, 5: 46.7, 4: 46.2).
#ifndef CLB_F16N_MINB
#define CLB_F16N_MINB 5
#endif
template <class P>
struct Step2MinBlocks {
    static constexpr int value = CLB_F16N_MINB;
};
#ifndef CLB_F16S_MINB
#define CLB_F16S_MINB 7
#endif
template <class L>
struct Step2MinBlocks<StoreH16T<L>> {
    static constexpr int value = CLB_F16S_MINB;
};

// OUTER: the pair tiles cover only the rows 0 and ny - 1 (thread rows 0 and
// 1 of one band of tiles), the other rows' interior pairs being taken by the
// TMA-fed kernel.
template <class P, bool SHIFT, bool FORCH, bool OUTER = false>
__global__ void __launch_bounds__(128, Step2MinBlocks<P>::value)
    k_step2(const BufT<typename P::S> in, const BufT<typename P::S> out,
                                                  const AuxT<float> A, const KParamsT<float> K, int tiles_x,
                                                  int n_tiles) {
    const int b = blockIdx.x;
    if (b < n_tiles) {
        const int x0 = 2 * ((b % tiles_x) * blockDim.x + threadIdx.x);
        int y = (b / tiles_x) * blockDim.y + threadIdx.y;
        if constexpr (OUTER) {
            // thread row 0 takes row 0 and thread row 1 row ny - 1; a block
            // of one thread row (small grids) takes both in turn
            if (threadIdx.y > 1) return;
            if (blockDim.y == 1 && interior_pair(K.g, x0, 0)) step_pair_interior<P, SHIFT, FORCH>(in, out, A, K, x0, 0);
            y = (threadIdx.y == 0 && blockDim.y > 1) ? 0 : K.g.ny - 1;
        }
        if (y >= K.g.ny || !interior_pair(K.g, x0, y)) return;
        step_pair_interior<P, SHIFT, FORCH>(in, out, A, K, x0, y);
    } else {
        const long long i = (long long)(b - n_tiles) * (blockDim.x * blockDim.y) + threadIdx.y * blockDim.x +
                            threadIdx.x;
        if (i >= edge_count(K.g)) return;
        int x, y;
        edge_node(K.g, i, x, y);
        step_node<P, SHIFT, FORCH>(in, out, A, K, x, y);
    }
}

// ---------------------------------------------------------------- batches
// One case of a batch: parameters, auxiliary pointers and both buffers.
template <typename R, typename S>
struct CaseT {
    KParamsT<R> K;
    AuxT<R> A;
    BufT<S> b[2];
    int flip;       // the case's current buffer is b[par ^ flip] (par: the batch's parity)
    int pad_;
};

// Independent cases advanced together.  `tiles` lists (case, x0, y0) in
// case order; a block takes the contiguous range [t0, t1), and its threads
// cover a (NPT * blockDim.x) x blockDim.y block of nodes at each tile (NPT =
// nodes per thread: 2 for the FP16 forms, 1 for FP64).  The case descriptor
// is staged in shared memory (raw) whenever the case changes.
template <class P, int NPT, bool SHIFT, bool FORCH>
__device__ __forceinline__ void batch_tiles(const CaseT<typename P::R, typename P::S>* __restrict__ cases,
                                            const int4* __restrict__ tiles, int t0, int t1, int par,
                                            unsigned char* raw, int& cur) {
    using C = CaseT<typename P::R, typename P::S>;
    C& sc = *reinterpret_cast<C*>(raw);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthr = blockDim.x * blockDim.y;
    for (int t = t0; t < t1; ++t) {
        const int4 tl = __ldg(tiles + t);
        if (tl.x != cur) {
            __syncthreads();
            const unsigned* src = reinterpret_cast<const unsigned*>(cases + tl.x);
            unsigned* dst = reinterpret_cast<unsigned*>(raw);
            for (int w = tid; w < (int)(sizeof(C) / 4); w += nthr) dst[w] = __ldg(src + w);
            __syncthreads();
            cur = tl.x;
        }
        const int x = tl.y + NPT * threadIdx.x, y = tl.z + threadIdx.y;
        if (x < sc.K.g.nx && y < sc.K.g.ny) {
            if constexpr (NPT == 2)
                step_pair<P, SHIFT, FORCH>(sc.b[par ^ sc.flip], sc.b[1 - (par ^ sc.flip)], sc.A, sc.K, x, y);
            else
                step_node<P, SHIFT, FORCH>(sc.b[par ^ sc.flip], sc.b[1 - (par ^ sc.flip)], sc.A, sc.K, x, y);
        }
    }
}

// Resident 128-thread blocks per SM the batch kernels are compiled for.
#ifndef CLB_BATCH_MINB
#define CLB_BATCH_MINB 4
#endif

// One step per launch: block b owns tiles [b * per_cta, (b + 1) * per_cta).
template <class P, int NPT, bool SHIFT, bool FORCH>
__global__ void __launch_bounds__(128, CLB_BATCH_MINB) k_step_batch(const CaseT<typename P::R, typename P::S>* __restrict__ cases,
                                                       const int4* __restrict__ tiles, int ntiles, int per_cta,
                                                       int par) {
    __shared__ __align__(16) unsigned char raw[sizeof(CaseT<typename P::R, typename P::S>)];
    const int t0 = blockIdx.x * per_cta;
    int cur = -1;
    batch_tiles<P, NPT, SHIFT, FORCH>(cases, tiles, t0, min(t0 + per_cta, ntiles), par, raw, cur);
}

// Interior pair tiles of a batch (the FP16 forms, graph mode): `tiles` lists
// (case, x0, y0) of tiles that lie in the interior-pair region of their case
// (x0 >= 2, rows inside the walls), so every thread runs the packed interior
// step and no thread carries the edge code; threads past the region's far
// edges skip.  Edge nodes go to k_step_batch_edge.
#ifndef CLB_BATCH_INT_MINB
#define CLB_BATCH_INT_MINB 5
#endif
// Loads case c's descriptor into the block's shared copy.
template <class C>
__device__ __forceinline__ void load_case(const C* __restrict__ cases, int c, unsigned char* raw) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthr = blockDim.x * blockDim.y;
    const unsigned* src = reinterpret_cast<const unsigned*>(cases + c);
    unsigned* dst = reinterpret_cast<unsigned*>(raw);
    for (int w = tid; w < (int)(sizeof(C) / 4); w += nthr) dst[w] = __ldg(src + w);
}

// Interior-pair tiles [t0, t1) of `tiles` (see k_step_batch_int).
template <class P, bool SHIFT, bool FORCH>
__device__ __forceinline__ void batch_int_tiles(const CaseT<typename P::R, typename P::S>* __restrict__ cases,
                                                const int4* __restrict__ tiles, int t0, int t1, int par,
                                                unsigned char* raw) {
    using C = CaseT<typename P::R, typename P::S>;
    C& sc = *reinterpret_cast<C*>(raw);
    int cur = -1;
    for (int t = t0; t < t1; ++t) {
        const int4 tl = __ldg(tiles + t);
        if (tl.x != cur) {
            __syncthreads();
            load_case(cases, tl.x, raw);
            __syncthreads();
            cur = tl.x;
        }
        const int x0 = tl.y + 2 * threadIdx.x, y = tl.z + threadIdx.y;
        const int y_hi = sc.K.g.wall_y ? sc.K.g.ny - 2 : sc.K.g.ny - 1;
        if (x0 + 2 < sc.K.g.nx && y <= y_hi) {
            const int b = par ^ sc.flip;
            step_pair_interior<P, SHIFT, FORCH>(sc.b[b], sc.b[1 - b], sc.A, sc.K, x0, y);
        }
    }
}

// One chunk (case, first edge index, count <= threads of the block) of edge
// nodes, one per thread (see k_step_batch_edge).
template <class P, bool SHIFT, bool FORCH>
__device__ __forceinline__ void batch_edge_chunk(const CaseT<typename P::R, typename P::S>* __restrict__ cases,
                                                 int4 ch, int par, unsigned char* raw) {
    using C = CaseT<typename P::R, typename P::S>;
    C& sc = *reinterpret_cast<C*>(raw);
    load_case(cases, ch.x, raw);
    __syncthreads();
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if (tid >= ch.z) return;
    int x, y;
    edge_node(sc.K.g, (long long)ch.y + tid, x, y);
    const int b = par ^ sc.flip;
    step_node<P, SHIFT, FORCH>(sc.b[b], sc.b[1 - b], sc.A, sc.K, x, y);
}

template <class P, bool SHIFT, bool FORCH>
__global__ void __launch_bounds__(128, CLB_BATCH_INT_MINB)
    k_step_batch_int(const CaseT<typename P::R, typename P::S>* __restrict__ cases, const int4* __restrict__ tiles,
                     int ntiles, int per_cta, int par) {
    __shared__ __align__(16) unsigned char raw[sizeof(CaseT<typename P::R, typename P::S>)];
    const int t0 = blockIdx.x * per_cta;
    batch_int_tiles<P, SHIFT, FORCH>(cases, tiles, t0, min(t0 + per_cta, ntiles), par, raw);
}

// Edge nodes of a batch (the nodes k_step2 leaves to its per-node path):
// `chunks` lists (case, first edge index, count) of at most blockDim nodes.
template <class P, bool SHIFT, bool FORCH>
__global__ void __launch_bounds__(128, 4)
    k_step_batch_edge(const CaseT<typename P::R, typename P::S>* __restrict__ cases, const int4* __restrict__ chunks,
                      int par) {
    __shared__ __align__(16) unsigned char raw[sizeof(CaseT<typename P::R, typename P::S>)];
    batch_edge_chunk<P, SHIFT, FORCH>(cases, __ldg(chunks + blockIdx.x), par, raw);
}

// Both in one launch: block i takes work[i] = (0, first tile) -- per_cta
// interior-pair tiles -- or (1, edge chunk).  The host orders the list so
// that each edge chunk follows the interior block that covers its last row:
// its column accesses (2 bytes of every 32-byte sector) then find the
// sectors they share with the neighbouring interior nodes in L2.  In a
// launch of their own the edge nodes fetched ~13x their bytes from DRAM.
// The kernel's registers are those of its larger path (the per-node edge
// step): 4 blocks per SM, where the interior kernel alone runs 5; capped at
// 5 it spills, and measured slower (36.4 against 37.9 GLUPS on 512 cases).
#ifndef CLB_BATCH_MIX_MINB
#define CLB_BATCH_MIX_MINB 4
#endif
template <class P, bool SHIFT, bool FORCH>
__global__ void __launch_bounds__(128, CLB_BATCH_MIX_MINB)
    k_step_batch_mix(const CaseT<typename P::R, typename P::S>* __restrict__ cases, const int4* __restrict__ work,
                     const int4* __restrict__ tiles, int ntiles, int per_cta, const int4* __restrict__ chunks, int par) {
    __shared__ __align__(16) unsigned char raw[sizeof(CaseT<typename P::R, typename P::S>)];
    const int4 w = __ldg(work + blockIdx.x);
    if (w.x == 0) batch_int_tiles<P, SHIFT, FORCH>(cases, tiles, w.y, min(w.y + per_cta, ntiles), par, raw);
    else batch_edge_chunk<P, SHIFT, FORCH>(cases, __ldg(chunks + w.y), par, raw);
}

// Grid barrier and work counters of the persistent batch launch, in device
// memory.  `arrived` counts block arrivals and next[s & 1] hands out the
// tiles of step s (both cleared before every launch; next[(s + 1) & 1] is
// cleared again by block 0 during step s, before it arrives); `failed` is
// set by a block whose wait gave up and stays set until the host reads and
// clears it.
struct GridBarrier {
    unsigned arrived;
    unsigned next[2];
    unsigned failed;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Block-wide: all blocks of the launch (plus `extra` that do not exist, for
// the failure-path test) arrive for step `step`; false if the wait gave up
// after `limit` SM clock cycles or another block had given up.  The
// __threadfence before arriving publishes this block's stores of the step,
// the acquiring load and the fence after the wait make the other blocks'
// stores visible (loads of the next step go to L2: LdCG).
__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, int step, int extra, long long limit, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        __threadfence();
        atomicAdd(&bar->arrived, 1u);
        const unsigned target = (unsigned)(step + 1) * (unsigned)(gridDim.x + extra);
        int ok = 1;
        const long long t0 = clock64();
        while (ld_acquire_gpu(&bar->arrived) < target) {
            if (ld_acquire_gpu(&bar->failed)) { ok = 0; break; }
            if (clock64() - t0 > limit) {
                atomicExch(&bar->failed, 1u);
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Persistent form: one cooperative launch (every block resident) advances
// the batch `nsteps` steps.  Within a step the blocks claim `chunk` tiles
// at a time from a counter (the tiles cost unequal amounts: wall tiles,
// ragged edges), and a bounded grid barrier separates the steps.  A barrier
// that gives up sets bar->failed and every block returns; the host reports
// CLB_ERR_TIMEOUT.
template <class P, int NPT, bool SHIFT, bool FORCH>
__global__ void __launch_bounds__(128, CLB_BATCH_MINB)
    k_step_batch_persist(const CaseT<typename P::R, typename P::S>* __restrict__ cases,
                         const int4* __restrict__ tiles, int ntiles, int chunk, int par0, int nsteps,
                         GridBarrier* bar, int extra, long long limit) {
    __shared__ __align__(16) unsigned char raw[sizeof(CaseT<typename P::R, typename P::S>)];
    __shared__ int s_ok, s_t;
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    int cur = -1;
    for (int step = 0; step < nsteps; ++step) {
        if (lead && blockIdx.x == 0) bar->next[(step + 1) & 1] = 0u;   // published by the barrier below
        while (true) {
            if (lead) s_t = (int)atomicAdd(&bar->next[step & 1], (unsigned)chunk);
            __syncthreads();
            const int t0 = s_t;
            __syncthreads();
            if (t0 >= ntiles) break;
            batch_tiles<P, NPT, SHIFT, FORCH>(cases, tiles, t0, min(t0 + chunk, ntiles), par0 ^ (step & 1), raw, cur);
        }
        if (step + 1 < nsteps || extra > 0)
            if (!grid_barrier(bar, step, extra, limit, &s_ok)) return;
    }
}

// Macroscopic fields at the current time level (dense ny*nx FP64 outputs),
// and (bad not NULL) the first node whose fields are not all finite.
template <class P, bool FORCH>
__global__ void k_macros(const BufT<typename P::S> in, const AuxT<typename P::R> A,
                         const KParamsT<typename P::R> K, double* __restrict__ orho, double* __restrict__ oux,
                         double* __restrict__ ouy, double* __restrict__ oT, unsigned long long* __restrict__ bad) {
    using R = typename P::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= K.g.nx || y >= K.g.ny) return;
    const long long n = (long long)y * K.g.nx + x;
    const CoefT<R> c = P::template coef<FORCH>(A, K, x, y);
    R f[9], g[5], rho, X, Y, T, Tt, hFx, hFy, n0;
    Mom9T<R> k;
    node_state<P, FORCH>(as_const(in), A, K, x, y, c, f, g, k, rho, X, Y, T, Tt, hFx, hFy, n0);
    if (orho) orho[n] = (double)rho;
    if (oux) oux[n] = (double)X;
    if (ouy) ouy[n] = (double)Y;
    if (oT) oT[n] = (double)T;
    // the smallest index of a node with a non-finite value (bad starts at ~0)
    if (bad && !(isfinite((double)rho) && isfinite((double)X) && isfinite((double)Y) && isfinite((double)T)))
        atomicMin(bad, (unsigned long long)n);
}

// Post-collision buffers whose pull reproduces the local equilibria of the
// given fields: slot i of node y holds f_i^eq of the node y + e_i that
// pulls it (periodic wrap; on a walled side the slot is never pulled and
// takes the node's own value).  The node's own fields are its baseline
// record in the FP16N form.
template <class P>
__global__ void k_set_fields(const BufT<typename P::S> out, const AuxT<typename P::R> A,
                             const double* __restrict__ rho, const double* __restrict__ ux,
                             const double* __restrict__ uy, const double* __restrict__ T,
                             const KParamsT<typename P::R> K) {
    using R = typename P::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= K.g.nx || y >= K.g.ny) return;
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    R f[9], g[5];
    // unrolled: each direction keeps one component of its neighbour's
    // equilibria, and the compiler drops the other eight (and four)
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int zx = x + ex[i], zy = y + ey[i];
        if (zx < 0 || zx >= K.g.nx) zx = K.g.wall_x ? x : wrap_hi(wrap_lo(zx, K.g.nx), K.g.nx);
        if (zy < 0 || zy >= K.g.ny) zy = K.g.wall_y ? y : wrap_hi(wrap_lo(zy, K.g.ny), K.g.ny);
        const long long z = (long long)zy * K.g.nx + zx;
        const R zr = (R)rho[z], zu = (R)ux[z], zv = (R)uy[z], zT = (R)T[z];
        R fe[9];
        feq9(zr, zu, zv, P::template coef<false>(A, K, zx, zy).ip, fe);
        f[i] = fe[i];
        if (i < 5) {
            R ge[5];
            if constexpr (P::kCentred)
                geq5c((R)(T[z] - (double)K.T0), zu, zv, K.p.sigma, K.p.cT2, R(K.T0), ge);
            else
                geq5(zT, zu, zv, K.p.sigma, K.p.cT2, ge);
            g[i] = ge[i];
        }
    }
    const long long n = (long long)y * K.g.nx + x;
    const R Tn = P::kCentred ? (R)(T[n] - (double)K.T0) : (R)T[n];   // the form's representation
    P::store(out, K, x, y, f, g, (R)rho[n], (R)ux[n], (R)uy[n], Tn, P::template coef<false>(A, K, x, y).ip,
             out.seq ? *out.seq : 0U);
}

// Four consecutive dense fields of n values set to constants.
__global__ void k_fill4(double* __restrict__ d, long long n, double a, double b, double c, double e) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    d[i] = a;
    d[n + i] = b;
    d[2 * n + i] = c;
    d[3 * n + i] = e;
}

// Per-node FP64 constants from the porosity (Eqs. 4, 5, 23) and the row's
// a_y - g beta T0 (ayg, one value per row).
__global__ void k_coef(const double* __restrict__ phi, const double* __restrict__ ayg, CoefT<double>* __restrict__ coef,
                       int nx, long long n, double nu, double K, double ax, double gbeta, int forch) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double p = phi[i], hp = 0.5 * p;
    CoefT<double> c;
    c.ip = 1.0 / p;
    c.hdar = hp * nu / K;
    c.l0 = 0.5 + 0.5 * c.hdar;                                   // Eq. 23
    c.l0sq = c.l0 * c.l0;
    if (forch) {
        const double Fphi = 1.75 / sqrt(150.0 * p * p * p);      // Ergun, Eq. 5
        c.aux = 0.5 * p * Fphi / sqrt(K);                         // l1 of Eq. 23
    } else {
        c.aux = 1.0 / (2.0 * c.l0);                               // 1 / (2 l0), Eq. 23
    }
    c.hgx = hp * ax;
    c.hgb = hp * gbeta;
    c.hgy = hp * ayg[i / nx];
    coef[i] = c;
}

// FP32 porosity (dense) for the FP16 rest-shifted form, or FP32 1/phi
// (pitched, px per row) for the FP16 equilibrium-shifted form.
__global__ void k_phi32(const double* __restrict__ phi, float* __restrict__ out, int nx, int ny, int px, int inv) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const long long y = i / nx, x = i - y * nx;
    if (inv) out[y * px + x] = (float)(1.0 / phi[i]);
    else out[i] = (float)phi[i];
}

}  // namespace clb
