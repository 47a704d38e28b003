// clb_f64.cuh -- FP64 device code of the coupled porous cascaded LB step.
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
// GB300 note: FP64 issues at a small fraction of the FP32 rate on this part,
// so this path is bound by FP64 instruction throughput, not by HBM.  The
// arithmetic is arranged to minimise FP64 operations per node: per-node
// constants (1/phi, phi/2, phi nu / K, l1 or 1/(2 l0)) are computed once at
// init, and only one division and (with the Forchheimer term) two square
// roots remain per node.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#ifndef CLB_HD
#define CLB_HD __host__ __device__ __forceinline__
#endif

namespace clb {

// Per-node constants derived from the porosity (Eqs. 4, 5, 23).
struct __align__(16) Coef {
    double ip;    // 1 / phi
    double hphi;  // phi / 2
    double dar;   // phi nu / K (Darcy coefficient of Eq. 4)
    double aux;   // Forchheimer: l1 = phi F_phi / (2 sqrt K); else 1 / (2 l0)
};

struct Geo {
    int nx, ny, px;       // grid and row pitch (elements)
    long long plane;      // px * ny
    int wall_x, wall_y;   // W/E resp. S/N are walls
};

struct Bnd {
    double uw[4], vw[4], Tw[4];
    int iso[4];
};

struct Phys {
    double ax, gbeta, inv_sigma, cT2;   // a_x, g*beta, 1/sigma, c_sT^2
    double sv, s3, s4, om_a;            // relaxation rates, om_a = 1 - zeta_alpha
    double sp, sm;                      // (s_b + s_v)/2, (s_b - s_v)/2: the (k20, k02) block of Eq. 15
    double c6;                          // (1 - s3/2) / 3  (Eq. 11 rows 6, 7 with Eq. 17)
    double ca, cb8;                     // MRT variant: 1 - s_v/2, 1 - s4/2
};

struct KParams {
    Geo g;
    Bnd b;
    Phys p;
};

__device__ __forceinline__ int wrap_lo(int a, int n) { return a < 0 ? a + n : a; }
__device__ __forceinline__ int wrap_hi(int a, int n) { return a >= n ? a - n : a; }

// f_i(x) = f*_i(x - e_i): the D2Q9 values streaming into (x, y).
__device__ __forceinline__ void pull9(const double* __restrict__ f, const Geo& G, int x, int y,
                                      double (&v)[9]) {
    const int xm = wrap_lo(x - 1, G.nx), xp = wrap_hi(x + 1, G.nx);
    const int ym = wrap_lo(y - 1, G.ny), yp = wrap_hi(y + 1, G.ny);
    const long long P = G.plane;
    const long long r0 = (long long)y * G.px, rm = (long long)ym * G.px, rp = (long long)yp * G.px;
    v[0] = __ldg(f + 0 * P + r0 + x);
    v[1] = __ldg(f + 1 * P + r0 + xm);
    v[2] = __ldg(f + 2 * P + rm + x);
    v[3] = __ldg(f + 3 * P + r0 + xp);
    v[4] = __ldg(f + 4 * P + rp + x);
    v[5] = __ldg(f + 5 * P + rm + xm);
    v[6] = __ldg(f + 6 * P + rm + xp);
    v[7] = __ldg(f + 7 * P + rp + xp);
    v[8] = __ldg(f + 8 * P + rp + xm);
}

__device__ __forceinline__ void pull5(const double* __restrict__ g, const Geo& G, int x, int y,
                                      double (&v)[5]) {
    const int xm = wrap_lo(x - 1, G.nx), xp = wrap_hi(x + 1, G.nx);
    const int ym = wrap_lo(y - 1, G.ny), yp = wrap_hi(y + 1, G.ny);
    const long long P = G.plane;
    const long long r0 = (long long)y * G.px;
    v[0] = __ldg(g + 0 * P + r0 + x);
    v[1] = __ldg(g + 1 * P + r0 + xm);
    v[2] = __ldg(g + 2 * P + (long long)ym * G.px + x);
    v[3] = __ldg(g + 3 * P + r0 + xp);
    v[4] = __ldg(g + 4 * P + (long long)yp * G.px + x);
}

// Raw moments of Eq. 12, M f, with the shared partial sums of M's rows.
struct Mom9 {
    double rho, jx, jy, k20, k02, k11, k21, k12, k22;
};

CLB_HD Mom9 moments9(const double (&f)[9]) {
    const double a = f[5] + f[7], b = f[6] + f[8];
    const double c = f[5] - f[7], d = f[6] - f[8];
    const double s13 = f[1] + f[3], s24 = f[2] + f[4];
    Mom9 k;
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

// Macroscopic velocity by Eqs. 22-23 and force by Eq. 4 at a node with
// density rho, momentum j = sum e f and temperature T.
template <bool FORCH>
CLB_HD void macro_velocity(double rho, double jx, double jy, double T, double ayg,
                                               const Coef& c, const Phys& P, double& X, double& Y,
                                               double& Fx, double& Fy) {
    const double irho = 1.0 / rho;
    const double Gy = fma(P.gbeta, T, ayg);           // a_y + g beta (T - T0), T0 folded into ayg
    const double hGx = c.hphi * P.ax, hGy = c.hphi * Gy;
    const double vx = fma(jx, irho, hGx), vy = fma(jy, irho, hGy);
    double cF;
    if (FORCH) {
        const double l0 = fma(0.25, c.dar, 0.5);
        const double vm = sqrt(fma(vx, vx, vy * vy));
        const double den = l0 + sqrt(fma(c.aux, vm, l0 * l0));
        const double inv = 1.0 / den;
        X = vx * inv;
        Y = vy * inv;
        cF = fma(2.0 * c.aux, vm * inv, c.dar);       // phi nu/K + phi F_phi/sqrt(K) |u|
    } else {
        X = vx * c.aux;
        Y = vy * c.aux;
        cF = c.dar;
    }
    Fx = fma(-cF, X, hGx + hGx);
    Fy = fma(-cF, Y, hGy + hGy);
}

// Porous flow equilibrium f^eq = M^-1 m^eq (Eq. 19).
CLB_HD void feq9(double rho, double X, double Y, double ip, double (&fe)[9]) {
    const double X2 = X * X, Y2 = Y * Y;
    const double r3 = rho * (1.0 / 3.0);
    const double m1 = rho * X, m2 = rho * Y;
    const double m3 = fma(m1 * ip, X, r3);
    const double m4 = fma(m2 * ip, Y, r3);
    const double m5 = m1 * Y * ip;
    const double m6 = fma(m1 * ip, X * Y, r3 * Y);
    const double m7 = fma(m2 * ip, X * Y, r3 * X);
    const double m8 = rho * (1.0 / 9.0) + r3 * ip * (X2 + Y2) + rho * X2 * Y2 * ip * ip;
    fe[0] = rho - m3 - m4 + m8;
    fe[1] = 0.5 * (m1 + m3 - m7 - m8);
    fe[2] = 0.5 * (m2 + m4 - m6 - m8);
    fe[3] = 0.5 * (-m1 + m3 + m7 - m8);
    fe[4] = 0.5 * (-m2 + m4 + m6 - m8);
    fe[5] = 0.25 * (m5 + m6 + m7 + m8);
    fe[6] = 0.25 * (-m5 + m6 - m7 + m8);
    fe[7] = 0.25 * (m5 - m6 - m7 + m8);
    fe[8] = 0.25 * (-m5 - m6 + m7 + m8);
}

// Thermal equilibrium g^eq = M_T^-1 n^eq (Eq. 33; equals Eq. 34).
CLB_HD void geq5(double T, double X, double Y, double sigma, double cT2,
                                     double (&ge)[5]) {
    const double n1 = X * T, n2 = Y * T;
    const double n3 = fma(X, n1, cT2 * T), n4 = fma(Y, n2, cT2 * T);
    ge[0] = sigma * T - n3 - n4;
    ge[1] = 0.5 * (n1 + n3);
    ge[2] = 0.5 * (n2 + n4);
    ge[3] = 0.5 * (n3 - n1);
    ge[4] = 0.5 * (n4 - n2);
}

// Flow collision (Eq. 11) in delta form; see the file comment.
template <bool SHIFT>
CLB_HD void collide9(double (&f)[9], const Mom9& k, double rho, double X, double Y,
                                         double Fx, double Fy, double ip, const Phys& P) {
    const double rFx = rho * Fx, rFy = rho * Fy;
    const double px = fma(rho, X, -k.jx), py = fma(rho, Y, -k.jy);   // -(k~10), -(k~01)
    const double X2 = X * X, Y2 = Y * Y, XY = X * Y;
    const double X2p = X + X, Y2p = Y + Y, XY4 = 4.0 * XY;
    const double r3 = rho * (1.0 / 3.0), r9 = rho * (1.0 / 9.0);
    const double D1 = fma(0.5, rFx, px);
    const double D2 = fma(0.5, rFy, py);
    double r3v, r4v, r5v, r6v, r7v, r8v;
    if (SHIFT) {
        // central moments m~3..m~8 = rows 3..8 of N (Eq. 14) times m
        const double ipX = ip * X, ipY = ip * Y;
        const double t = px - k.jx, tp = py - k.jy;        // rho X - 2 jx, rho Y - 2 jy
        const double Xjy = X * k.jy, Yjx = Y * k.jx;
        const double c3 = fma(ipX, t, k.k20);
        const double c4 = fma(ipY, tp, k.k02);
        const double c5 = fma(ip, fma(Y, px, -Xjy), k.k11);
        const double w = fma(-Y, t, Xjy);
        const double c6 = fma(ipX, w, fma(-Y, k.k20, fma(-X2p, k.k11, k.k21)));
        const double wp = fma(-X, tp, Yjx);
        const double c7 = fma(ipY, wp, fma(-X, k.k02, fma(-Y2p, k.k11, k.k12)));
        double A = Y2 * k.k20;
        A = fma(X2, k.k02, A);
        A = fma(XY4, k.k11, A);
        A = fma(-Y2p, k.k21, A);
        A = fma(-X2p, k.k12, A);
        A = fma(-(ip * XY), w + Xjy, A);
        const double c8 = fma(ip, A, k.k22);
        // increments of Eq. 11 (Lambda of Eq. 15 with s_0 = s_1 = 1)
        const double e3 = r3 - c3, e4 = r3 - c4;
        const double D3 = fma(P.sp, e3, P.sm * e4);
        const double D4 = fma(P.sp, e4, P.sm * e3);
        const double D5 = -P.sv * c5;
        const double D6 = fma(-P.s3, c6, P.c6 * rFy);
        const double D7 = fma(-P.s3, c7, P.c6 * rFx);
        const double D8 = P.s4 * (r9 - c8);
        // back to raw moments: N^-1 Delta (Eq. A1), Delta_0 = 0
        const double ipX2 = ipX + ipX, ipY2 = ipY + ipY;
        r3v = fma(ipX2, D1, D3);
        r4v = fma(ipY2, D2, D4);
        r5v = fma(ipY, D1, fma(ipX, D2, D5));
        r6v = fma(ipX, fma(Y2p, D1, X * D2), fma(Y, D3, fma(X2p, D5, D6)));
        r7v = fma(ipY, fma(Y, D1, X2p * D2), fma(X, D4, fma(Y2p, D5, D7)));
        double B = Y2 * D3;
        B = fma(X2, D4, B);
        B = fma(XY4, D5, B);
        B = fma(Y2p, D6, B);
        B = fma(X2p, D7, B);
        B = fma(2.0 * ip * XY, fma(Y, D1, X * D2), B);
        r8v = fma(ip, B, D8);
    } else {
        // unit shift: relax raw moments towards Eq. 19's m^eq with Eq. 19's S
        const double ipr = ip * rho;
        const double meq3 = fma(ipr * X, X, r3), meq4 = fma(ipr * Y, Y, r3);
        const double meq5 = ipr * XY;
        const double meq6 = fma(ipr * X2, Y, r3 * Y), meq7 = fma(ipr * Y2, X, r3 * X);
        const double meq8 = r9 + r3 * ip * (X2 + Y2) + ipr * ip * X2 * Y2;
        const double S3 = 2.0 * ip * X * rFx, S4 = 2.0 * ip * Y * rFy;
        const double S5 = ip * fma(X, rFy, Y * rFx);
        const double S6 = fma(ip, fma(X2, rFy, 2.0 * XY * rFx), rFy * (1.0 / 3.0));
        const double S7 = fma(ip, fma(Y2, rFx, 2.0 * XY * rFy), rFx * (1.0 / 3.0));
        const double S8 = (2.0 / 3.0) * ip * fma(X, rFx, Y * rFy) + 2.0 * ip * ip * XY * fma(Y, rFx, X * rFy);
        // (k20, k02) block: -Lambda_b (m - m^eq) + (I - Lambda_b / 2) S
        const double d3 = k.k20 - meq3, d4 = k.k02 - meq4;
        r3v = -fma(P.sp, d3, P.sm * d4) + S3 - 0.5 * fma(P.sp, S3, P.sm * S4);
        r4v = -fma(P.sm, d3, P.sp * d4) + S4 - 0.5 * fma(P.sm, S3, P.sp * S4);
        r5v = fma(-P.sv, k.k11 - meq5, P.ca * S5);
        r6v = fma(-P.s3, k.k21 - meq6, 3.0 * P.c6 * S6);
        r7v = fma(-P.s3, k.k12 - meq7, 3.0 * P.c6 * S7);
        r8v = fma(-P.s4, k.k22 - meq8, P.cb8 * S8);
    }
    // f* = f + M^-1 r, r = (0, D1, D2, r3..r8)
    const double pa = r3v - r8v, qa = D1 - r7v;
    const double pb = r4v - r8v, qb = D2 - r6v;
    const double u1 = r8v + r5v, u2 = r8v - r5v, v1 = r6v + r7v, v2 = r6v - r7v;
    f[0] += (r8v - r3v) - r4v;
    f[1] = fma(0.5, pa + qa, f[1]);
    f[3] = fma(0.5, pa - qa, f[3]);
    f[2] = fma(0.5, pb + qb, f[2]);
    f[4] = fma(0.5, pb - qb, f[4]);
    f[5] = fma(0.25, u1 + v1, f[5]);
    f[7] = fma(0.25, u1 - v1, f[7]);
    f[6] = fma(0.25, u2 + v2, f[6]);
    f[8] = fma(0.25, u2 - v2, f[8]);
}

// Temperature collision (Eq. 28) with zeta_T = zeta_e = zeta_nu = 1:
// g* = M_T^-1 N_T^-1 n~*, n~* = (sigma T, (1 - zeta_a) n~1, (1 - zeta_a) n~2,
// c_sT^2 T, c_sT^2 T), where n~1 = n1 - u_x T (Eq. 31 with sigma T = n0).
// Back-shifting (N_T^-1) gives n1* = u_x T + n~1*, n3* = u_x^2 T + 2 u_x n~1*
// + c_sT^2 T.  The unit-shift variant relaxes the raw moments towards
// Eq. 33 instead: n1* as above, n3* = (c_sT^2 + u_x^2) T.
template <bool SHIFT>
CLB_HD void collide5(double (&g)[5], double n0, double T, double X, double Y, const Phys& P) {
    const double XT = X * T, YT = Y * T;
    const double c1 = P.om_a * ((g[1] - g[3]) - XT);   // (1 - zeta_a) n~1
    const double c2 = P.om_a * ((g[2] - g[4]) - YT);
    const double n1 = XT + c1, n2 = YT + c2;
    const double cT = P.cT2 * T;
    const double n3 = SHIFT ? fma(X + X, c1, fma(X, XT, cT)) : fma(X, XT, cT);
    const double n4 = SHIFT ? fma(Y + Y, c2, fma(Y, YT, cT)) : fma(Y, YT, cT);
    g[0] = (n0 - n3) - n4;
    g[1] = 0.5 * (n1 + n3);
    g[2] = 0.5 * (n2 + n4);
    g[3] = 0.5 * (n3 - n1);
    g[4] = 0.5 * (n4 - n2);
}

// Inward normal of a wall node and the sides that set its velocity and
// temperature.  Returns false for an interior node.
struct WallInfo {
    int dx, dy, su, st;
};

__device__ __forceinline__ bool wall_info(const Geo& G, const Bnd& B, int x, int y, WallInfo& w) {
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
template <bool FORCH>
__device__ __forceinline__ void wall_state(const double* __restrict__ fin, const double* __restrict__ gin,
                                           const Coef* __restrict__ coef, const double* __restrict__ ayg,
                                           const KParams& K, int x, int y, const WallInfo& w,
                                           double (&f)[9], double (&g)[5], double& rho, double& X,
                                           double& Y, double& T, double& n0) {
    const int sx = x + w.dx, sy = y + w.dy;
    double fs[9], gs[5];
    pull9(fin, K.g, sx, sy, fs);
    pull5(gin, K.g, sx, sy, gs);
    const Mom9 ks = moments9(fs);
    const double Ts = ((gs[0] + gs[1]) + (gs[2] + gs[3]) + gs[4]) * K.p.inv_sigma;
    const Coef cs = coef[(long long)sy * K.g.nx + sx];
    double Xs, Ys, Fxs, Fys;
    macro_velocity<FORCH>(ks.rho, ks.jx, ks.jy, Ts, ayg[sy], cs, K.p, Xs, Ys, Fxs, Fys);
    double Tb;
    if (w.st >= 0) {
        Tb = K.b.Tw[w.st];
    } else {
        double gss[5];
        pull5(gin, K.g, x + 2 * w.dx, y + 2 * w.dy, gss);
        const double Tss = ((gss[0] + gss[1]) + (gss[2] + gss[3]) + gss[4]) * K.p.inv_sigma;
        Tb = (4.0 * Ts - Tss) * (1.0 / 3.0);
    }
    const double uw = K.b.uw[w.su], vw = K.b.vw[w.su];
    const double ipb = coef[(long long)y * K.g.nx + x].ip;
    double fb[9], fe[9];
    feq9(ks.rho, uw, vw, ipb, fb);
    feq9(ks.rho, Xs, Ys, cs.ip, fe);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = fb[i] + (fs[i] - fe[i]);
    const double sigma = 1.0 / K.p.inv_sigma;
    double gb[5], ge[5];
    geq5(Tb, uw, vw, sigma, K.p.cT2, gb);
    geq5(Ts, Xs, Ys, sigma, K.p.cT2, ge);
#pragma unroll
    for (int i = 0; i < 5; ++i) g[i] = gb[i] + (gs[i] - ge[i]);
    rho = ks.rho;
    X = uw;
    Y = vw;
    T = Tb;
    n0 = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
}

// Force of Eq. 4 at a node whose velocity is imposed (wall nodes).
template <bool FORCH>
CLB_HD void force_at(double X, double Y, double T, double ayg, const Coef& c,
                                         const Phys& P, double& Fx, double& Fy) {
    const double Gy = fma(P.gbeta, T, ayg);
    double cF = c.dar;
    if (FORCH) cF = fma(2.0 * c.aux, sqrt(fma(X, X, Y * Y)), c.dar);
    Fx = fma(-cF, X, 2.0 * c.hphi * P.ax);
    Fy = fma(-cF, Y, 2.0 * c.hphi * Gy);
}

// ---------------------------------------------------------------- kernels
template <bool SHIFT, bool FORCH>
__global__ void __launch_bounds__(256) k_step_f64(const double* __restrict__ fin,
                                                  const double* __restrict__ gin,
                                                  double* __restrict__ fout, double* __restrict__ gout,
                                                  const Coef* __restrict__ coef,
                                                  const double* __restrict__ ayg, const KParams K) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= K.g.nx || y >= K.g.ny) return;
    const Coef c = coef[(long long)y * K.g.nx + x];
    double f[9], g[5];
    double rho, X, Y, T, Fx, Fy, n0;
    Mom9 k;
    WallInfo w;
    if (!wall_info(K.g, K.b, x, y, w)) {
        pull9(fin, K.g, x, y, f);
        pull5(gin, K.g, x, y, g);
        k = moments9(f);
        n0 = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
        T = n0 * K.p.inv_sigma;
        rho = k.rho;
        macro_velocity<FORCH>(rho, k.jx, k.jy, T, ayg[y], c, K.p, X, Y, Fx, Fy);
    } else {
        wall_state<FORCH>(fin, gin, coef, ayg, K, x, y, w, f, g, rho, X, Y, T, n0);
        k = moments9(f);
        force_at<FORCH>(X, Y, T, ayg[y], c, K.p, Fx, Fy);
    }
    collide9<SHIFT>(f, k, rho, X, Y, Fx, Fy, c.ip, K.p);
    collide5<SHIFT>(g, n0, T, X, Y, K.p);
    const long long o = (long long)y * K.g.px + x;
    const long long P = K.g.plane;
#pragma unroll
    for (int i = 0; i < 9; ++i) fout[i * P + o] = f[i];
#pragma unroll
    for (int i = 0; i < 5; ++i) gout[i * P + o] = g[i];
}

// Macroscopic fields at the current time level (dense ny*nx outputs).
template <bool FORCH>
__global__ void k_macros_f64(const double* __restrict__ fin, const double* __restrict__ gin,
                             const Coef* __restrict__ coef, const double* __restrict__ ayg,
                             const KParams K, double* __restrict__ orho, double* __restrict__ oux,
                             double* __restrict__ ouy, double* __restrict__ oT) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= K.g.nx || y >= K.g.ny) return;
    const long long n = (long long)y * K.g.nx + x;
    double f[9], g[5], rho, X, Y, T, n0;
    WallInfo w;
    if (!wall_info(K.g, K.b, x, y, w)) {
        pull9(fin, K.g, x, y, f);
        pull5(gin, K.g, x, y, g);
        const Mom9 k = moments9(f);
        T = (((g[0] + g[1]) + (g[2] + g[3])) + g[4]) * K.p.inv_sigma;
        rho = k.rho;
        double Fx, Fy;
        macro_velocity<FORCH>(rho, k.jx, k.jy, T, ayg[y], coef[n], K.p, X, Y, Fx, Fy);
    } else {
        wall_state<FORCH>(fin, gin, coef, ayg, K, x, y, w, f, g, rho, X, Y, T, n0);
    }
    if (orho) orho[n] = rho;
    if (oux) oux[n] = X;
    if (ouy) ouy[n] = Y;
    if (oT) oT[n] = T;
}

// Post-collision buffers whose pull reproduces the local equilibria of the
// given fields: slot i of node y holds f_i^eq of the node y + e_i that
// pulls it (periodic wrap; on a walled side the slot is never pulled and
// takes the node's own value).
__global__ void k_set_fields_f64(double* __restrict__ f, double* __restrict__ g,
                                 const Coef* __restrict__ coef, const double* __restrict__ rho,
                                 const double* __restrict__ ux, const double* __restrict__ uy,
                                 const double* __restrict__ T, double sigma, const KParams K) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= K.g.nx || y >= K.g.ny) return;
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const long long o = (long long)y * K.g.px + x;
#pragma unroll 1
    for (int i = 0; i < 9; ++i) {
        int zx = x + ex[i], zy = y + ey[i];
        if (zx < 0 || zx >= K.g.nx) zx = K.g.wall_x ? x : wrap_hi(wrap_lo(zx, K.g.nx), K.g.nx);
        if (zy < 0 || zy >= K.g.ny) zy = K.g.wall_y ? y : wrap_hi(wrap_lo(zy, K.g.ny), K.g.ny);
        const long long z = (long long)zy * K.g.nx + zx;
        double fe[9];
        feq9(rho[z], ux[z], uy[z], coef[z].ip, fe);
        f[i * K.g.plane + o] = fe[i];
        if (i < 5) {
            double ge[5];
            geq5(T[z], ux[z], uy[z], sigma, K.p.cT2, ge);
            g[i * K.g.plane + o] = ge[i];
        }
    }
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

// Per-node constants from the porosity (Eqs. 4, 5, 23).
__global__ void k_coef(const double* __restrict__ phi, Coef* __restrict__ coef, long long n, double nu,
                       double K, int forch) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double p = phi[i];
    Coef c;
    c.ip = 1.0 / p;
    c.hphi = 0.5 * p;
    c.dar = p * nu / K;
    if (forch) {
        const double Fphi = 1.75 / sqrt(150.0 * p * p * p);      // Ergun, Eq. 5
        c.aux = 0.5 * p * Fphi / sqrt(K);                         // l1 of Eq. 23
    } else {
        c.aux = 1.0 / (1.0 + 0.5 * c.dar);                        // 1 / (2 l0), Eq. 23
    }
    coef[i] = c;
}

}  // namespace clb
