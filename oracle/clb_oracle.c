/*
 * clb_oracle.c -- plain, slow FP64 CPU oracle for the REV-scale cascaded
 * lattice Boltzmann (CLB) method of Feng, Liu & He, "Numerical simulations of
 * convection heat transfer in porous media using a cascaded lattice Boltzmann
 * method" (arXiv:2110.05943).
 *
 * TEST INFRASTRUCTURE.  This file exists only so that tests/, the smoke check
 * in __graft_entry__ and the cpu_baseline leg of bench.py can check the CUDA
 * path against an independent restatement of the paper.  No product code may
 * include, link or call it, and it shares no source with the CUDA library.
 *
 * Everything is computed the literal way, in the paper's order and notation:
 *   - dense 9x9 and 5x5 matrix products for M (Eq. 13), N (Eq. 14),
 *     Lambda (Eq. 15), N^-1 (Eq. A1), M^-1 (numeric Gauss-Jordan inverse),
 *     M_T (Eq. 30), N_T (Eq. 31), Q (Eq. 28), N_T^-1 and M_T^-1;
 *   - equilibria and forcing from Eq. 16, 17, 19 (flow) and Eq. 32, 33
 *     (temperature), built as written;
 *   - macroscopic quantities from Eqs. 20, 22, 23, 36 and the force of Eq. 4
 *     with the Ergun inertia coefficient of Eq. 5;
 *   - collision Eq. 11 / Eq. 28, streaming Eq. 18 / Eq. 35 as a push from
 *     each node to its neighbour;
 *   - walls by non-equilibrium extrapolation (Sec. 3, cited there as [55]);
 *     the paper does not spell that scheme out, so the reading used here is:
 *     after streaming, a wall node b with inward fluid neighbour x_f gets
 *       f_i(b) = f_i^eq(rho_f, u_w; phi_b) + f_i(x_f) - f_i^eq(rho_f, u_f; phi_f)
 *       g_i(b) = g_i^eq(T_b, u_w)          + g_i(x_f) - g_i^eq(T_f, u_f)
 *     with T_b = T_w (isothermal) or (4 T_f - T_ff)/3 (adiabatic, second
 *     order), and b is then collided like any node with rho = rho_f, u = u_w,
 *     T = T_b.  At a corner x_f is the diagonal neighbour, the velocity of
 *     the vertical (W/E) wall is used, and an isothermal wall wins over an
 *     adiabatic one (vertical first).
 *
 * State convention: the oracle stores the pre-collision distributions
 * f(x, t), g(x, t) of every node, array-of-structures f[(y*nx + x)*9 + i].
 * Wall nodes always hold their reconstructed values.
 *
 * parity unpinned: none -- every routine here is pinned by a test in
 * tests/test_oracle_*.py (matrix identities, closed-form channel profiles,
 * conservation, decay rates, brute-force central moments).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction,
 * so the arithmetic is exactly the C source's order).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- lattices */
/* D2Q9 velocities of Eq. 6 (c = 1): rest, four axis, four diagonal. */
static const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* Moment exponents (m, n) of the simplified set of Eq. 9. */
static const int MM9[9] = {0, 1, 0, 2, 0, 1, 2, 1, 2};
static const int MN9[9] = {0, 0, 1, 0, 2, 1, 1, 2, 2};
/* D2Q5 uses velocities 0..4 of Eq. 6 and the moment set of Eq. 26. */
static const int MM5[5] = {0, 1, 0, 2, 0};
static const int MN5[5] = {0, 0, 1, 0, 2};

static double ipow(int b, int e) {
    double r = 1.0;
    for (int k = 0; k < e; ++k) r *= (double)b;
    return r;
}

/* M of Eqs. 7, 9, 12: row r = <f | e_x^m e_y^n>. */
void orc_matrix_M(double *M) {
    for (int r = 0; r < 9; ++r)
        for (int i = 0; i < 9; ++i) M[r * 9 + i] = ipow(EX9[i], MM9[r]) * ipow(EY9[i], MN9[r]);
}

/* M_T of Eqs. 24, 26, 29. */
void orc_matrix_MT(double *M) {
    for (int r = 0; r < 5; ++r)
        for (int i = 0; i < 5; ++i) M[r * 5 + i] = ipow(EX9[i], MM5[r]) * ipow(EY9[i], MN5[r]);
}

/* Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix.
 * Returns 0 on success, -1 if singular. */
int orc_invert(int n, const double *A, double *Ainv) {
    double a[81 * 2];
    int w = 2 * n;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < w; ++c) a[r * w + c] = (c < n) ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r * w + col]) > fabs(a[piv * w + col])) piv = r;
        if (a[piv * w + col] == 0.0) return -1;
        if (piv != col)
            for (int c = 0; c < w; ++c) {
                double t = a[col * w + c];
                a[col * w + c] = a[piv * w + c];
                a[piv * w + c] = t;
            }
        double p = a[col * w + col];
        for (int c = 0; c < w; ++c) a[col * w + c] /= p;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double m = a[r * w + col];
            if (m == 0.0) continue;
            for (int c = 0; c < w; ++c) a[r * w + c] -= m * a[col * w + c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = a[r * w + n + c];
    return 0;
}

/* Shift matrix N of Eq. 14 (porosity-aware), written entry by entry. */
void orc_matrix_N(double ux, double uy, double phi, double *N) {
    double p = phi, p2 = phi * phi;
    double x2 = ux * ux, y2 = uy * uy, xy = ux * uy;
    for (int k = 0; k < 81; ++k) N[k] = 0.0;
#define E(r, c) N[(r) * 9 + (c)]
    E(0, 0) = 1.0;
    E(1, 0) = -ux;            E(1, 1) = 1.0;
    E(2, 0) = -uy;            E(2, 2) = 1.0;
    E(3, 0) = x2 / p;         E(3, 1) = -2.0 * ux / p;  E(3, 3) = 1.0;
    E(4, 0) = y2 / p;         E(4, 2) = -2.0 * uy / p;  E(4, 4) = 1.0;
    E(5, 0) = xy / p;         E(5, 1) = -uy / p;        E(5, 2) = -ux / p;   E(5, 5) = 1.0;
    E(6, 0) = -x2 * uy / p;   E(6, 1) = 2.0 * xy / p;   E(6, 2) = x2 / p;
    E(6, 3) = -uy;            E(6, 5) = -2.0 * ux;      E(6, 6) = 1.0;
    E(7, 0) = -y2 * ux / p;   E(7, 1) = y2 / p;         E(7, 2) = 2.0 * xy / p;
    E(7, 4) = -ux;            E(7, 5) = -2.0 * uy;      E(7, 7) = 1.0;
    E(8, 0) = x2 * y2 / p2;   E(8, 1) = -2.0 * ux * y2 / p2; E(8, 2) = -2.0 * uy * x2 / p2;
    E(8, 3) = y2 / p;         E(8, 4) = x2 / p;         E(8, 5) = 4.0 * xy / p;
    E(8, 6) = -2.0 * uy / p;  E(8, 7) = -2.0 * ux / p;  E(8, 8) = 1.0;
#undef E
}

/* Inverse shift matrix N^-1 as printed in Appendix A (Eq. A1). */
void orc_matrix_Ninv(double ux, double uy, double phi, double *N) {
    double p = phi, p2 = phi * phi;
    double x2 = ux * ux, y2 = uy * uy, xy = ux * uy;
    for (int k = 0; k < 81; ++k) N[k] = 0.0;
#define E(r, c) N[(r) * 9 + (c)]
    E(0, 0) = 1.0;
    E(1, 0) = ux;             E(1, 1) = 1.0;
    E(2, 0) = uy;             E(2, 2) = 1.0;
    E(3, 0) = x2 / p;         E(3, 1) = 2.0 * ux / p;   E(3, 3) = 1.0;
    E(4, 0) = y2 / p;         E(4, 2) = 2.0 * uy / p;   E(4, 4) = 1.0;
    E(5, 0) = xy / p;         E(5, 1) = uy / p;         E(5, 2) = ux / p;    E(5, 5) = 1.0;
    E(6, 0) = x2 * uy / p;    E(6, 1) = 2.0 * xy / p;   E(6, 2) = x2 / p;
    E(6, 3) = uy;             E(6, 5) = 2.0 * ux;       E(6, 6) = 1.0;
    E(7, 0) = y2 * ux / p;    E(7, 1) = y2 / p;         E(7, 2) = 2.0 * xy / p;
    E(7, 4) = ux;             E(7, 5) = 2.0 * uy;       E(7, 7) = 1.0;
    E(8, 0) = x2 * y2 / p2;   E(8, 1) = 2.0 * ux * y2 / p2; E(8, 2) = 2.0 * uy * x2 / p2;
    E(8, 3) = y2 / p;         E(8, 4) = x2 / p;         E(8, 5) = 4.0 * xy / p;
    E(8, 6) = 2.0 * uy / p;   E(8, 7) = 2.0 * ux / p;   E(8, 8) = 1.0;
#undef E
}

/* Shift matrix N_T of Eq. 31 (heat-capacity-ratio-aware). */
void orc_matrix_NT(double ux, double uy, double sigma, double *N) {
    for (int k = 0; k < 25; ++k) N[k] = 0.0;
#define E(r, c) N[(r) * 5 + (c)]
    E(0, 0) = 1.0;
    E(1, 0) = -ux / sigma;       E(1, 1) = 1.0;
    E(2, 0) = -uy / sigma;       E(2, 2) = 1.0;
    E(3, 0) = ux * ux / sigma;   E(3, 1) = -2.0 * ux;  E(3, 3) = 1.0;
    E(4, 0) = uy * uy / sigma;   E(4, 2) = -2.0 * uy;  E(4, 4) = 1.0;
#undef E
}

/* N_T^-1.  The appendix breaks off after Eq. A1, so this inverse is derived
 * here by solving N_T X = I for the lower-triangular X (the test suite checks
 * N_T N_T^-1 = I). */
void orc_matrix_NTinv(double ux, double uy, double sigma, double *N) {
    for (int k = 0; k < 25; ++k) N[k] = 0.0;
#define E(r, c) N[(r) * 5 + (c)]
    E(0, 0) = 1.0;
    E(1, 0) = ux / sigma;        E(1, 1) = 1.0;
    E(2, 0) = uy / sigma;        E(2, 2) = 1.0;
    E(3, 0) = ux * ux / sigma;   E(3, 1) = 2.0 * ux;   E(3, 3) = 1.0;
    E(4, 0) = uy * uy / sigma;   E(4, 2) = 2.0 * uy;   E(4, 4) = 1.0;
#undef E
}

/* Relaxation matrix Lambda of Eq. 15, block diagonal, with
 * s+ = (s_b + s_v)/2 and s- = (s_b - s_v)/2 acting on (k20, k02). */
void orc_matrix_Lambda(double s0, double s1, double sb, double sv, double s3, double s4, double *L) {
    for (int k = 0; k < 81; ++k) L[k] = 0.0;
    double sp = 0.5 * (sb + sv), sm = 0.5 * (sb - sv);
    L[0 * 9 + 0] = s0;
    L[1 * 9 + 1] = s1;
    L[2 * 9 + 2] = s1;
    L[3 * 9 + 3] = sp; L[3 * 9 + 4] = sm;
    L[4 * 9 + 3] = sm; L[4 * 9 + 4] = sp;
    L[5 * 9 + 5] = sv;
    L[6 * 9 + 6] = s3;
    L[7 * 9 + 7] = s3;
    L[8 * 9 + 8] = s4;
}

/* Equilibrium central moments, Eq. 16 (c_s^2 = 1/3). */
void orc_meq_central(double rho, double *m) {
    double cs2 = 1.0 / 3.0;
    m[0] = rho; m[1] = 0.0; m[2] = 0.0; m[3] = rho * cs2; m[4] = rho * cs2;
    m[5] = 0.0; m[6] = 0.0; m[7] = 0.0; m[8] = rho * cs2 * cs2;
}

/* Central-moment forcing, Eq. 17. */
void orc_S_central(double rho, double Fx, double Fy, double *S) {
    double cs2 = 1.0 / 3.0;
    S[0] = 0.0; S[1] = rho * Fx; S[2] = rho * Fy; S[3] = 0.0; S[4] = 0.0; S[5] = 0.0;
    S[6] = cs2 * rho * Fy; S[7] = cs2 * rho * Fx; S[8] = 0.0;
}

/* Equilibrium raw moments, Eq. 19 (left vector). */
void orc_meq_raw(double rho, double ux, double uy, double phi, double *m) {
    double p = phi;
    m[0] = rho;
    m[1] = rho * ux;
    m[2] = rho * uy;
    m[3] = rho / 3.0 + rho * ux * ux / p;
    m[4] = rho / 3.0 + rho * uy * uy / p;
    m[5] = rho * ux * uy / p;
    m[6] = rho * uy / 3.0 + rho * ux * ux * uy / p;
    m[7] = rho * ux / 3.0 + rho * ux * uy * uy / p;
    m[8] = rho / 9.0 + rho * (ux * ux + uy * uy) / (3.0 * p) + rho * ux * ux * uy * uy / (p * p);
}

/* Raw-moment forcing, Eq. 19 (right vector). */
void orc_S_raw(double rho, double ux, double uy, double Fx, double Fy, double phi, double *S) {
    double p = phi;
    S[0] = 0.0;
    S[1] = rho * Fx;
    S[2] = rho * Fy;
    S[3] = 2.0 * rho * ux * Fx / p;
    S[4] = 2.0 * rho * uy * Fy / p;
    S[5] = rho * (ux * Fy + uy * Fx) / p;
    S[6] = rho * Fy / 3.0 + rho * Fy * ux * ux / p + 2.0 * rho * Fx * ux * uy / p;
    S[7] = rho * Fx / 3.0 + rho * Fx * uy * uy / p + 2.0 * rho * Fy * uy * ux / p;
    S[8] = (2.0 / 3.0) * rho * (ux * Fx + uy * Fy) / p + 2.0 * rho * Fx * ux * uy * uy / (p * p) +
           2.0 * rho * Fy * uy * ux * ux / (p * p);
}

/* Thermal equilibrium central moments, Eq. 32 (c_sT^2 = varpi/2). */
void orc_neq_central(double T, double sigma, double varpi, double *n) {
    double c2 = 0.5 * varpi;
    n[0] = sigma * T; n[1] = 0.0; n[2] = 0.0; n[3] = c2 * T; n[4] = c2 * T;
}

/* Thermal equilibrium raw moments, Eq. 33. */
void orc_neq_raw(double T, double ux, double uy, double sigma, double varpi, double *n) {
    double c2 = 0.5 * varpi;
    n[0] = sigma * T; n[1] = ux * T; n[2] = uy * T;
    n[3] = (c2 + ux * ux) * T; n[4] = (c2 + uy * uy) * T;
}

static void matvec(int n, const double *A, const double *x, double *y) {
    for (int r = 0; r < n; ++r) {
        double s = 0.0;
        for (int c = 0; c < n; ++c) s += A[r * n + c] * x[c];
        y[r] = s;
    }
}

/* Inertia coefficient of Eq. 5 (Ergun). */
double orc_ergun_Fphi(double phi) { return 1.75 / sqrt(150.0 * phi * phi * phi); }

/* ------------------------------------------------------------ configuration */
typedef struct {
    int nx, ny;
    int kind[4];              /* W, E, S, N: 0 periodic, 1 wall */
    double uw[4], vw[4];      /* wall velocity */
    int tdir[4];              /* 1 isothermal (Dirichlet), 0 adiabatic */
    double Tw[4];
    double nu, nu_e, K;       /* fluid and effective viscosity, permeability */
    double gbeta;             /* g*beta (lattice units); gravity along -y */
    double sigma, varpi, T0;
    double ax;                /* x component of the external acceleration a */
    double s0, s1, sb, sv, s3, s4;      /* Eq. 15 */
    double zT, za, ze, zn;              /* Eq. 28: zeta_T, zeta_alpha, zeta_e, zeta_nu */
    int forchheimer;          /* 1: F_phi from Eq. 5; 0: F_phi = 0 */
    int shift;                /* 1: N, N_T of Eq. 14/31; 0: unit shift (MRT limit) */
    int nthreads;
} orc_cfg;

typedef struct {
    orc_cfg c;
    double *phi, *ay;         /* porosity per node, a_y per row */
    double *f, *g, *fs, *gs;  /* pre-collision state and post-collision scratch */
    unsigned char *wall;      /* 1 for wall nodes */
    double *wrho, *wux, *wuy, *wT;   /* macroscopic values imposed at wall nodes */
    double M[81], Minv[81], MT[25], MTinv[25], L[81], Q[25];
} orc_t;

static int is_wall_node(const orc_cfg *c, int x, int y) {
    if (c->kind[0] && x == 0) return 1;
    if (c->kind[1] && x == c->nx - 1) return 1;
    if (c->kind[2] && y == 0) return 1;
    if (c->kind[3] && y == c->ny - 1) return 1;
    return 0;
}

/* Flow equilibrium f^eq = M^-1 m^eq (Eq. 19 and the text after it). */
static void feq_of(const orc_t *o, double rho, double ux, double uy, double phi, double *feq) {
    double m[9];
    orc_meq_raw(rho, ux, uy, phi, m);
    matvec(9, o->Minv, m, feq);
}

/* Thermal equilibrium g^eq = M_T^-1 n^eq (Eq. 33 and the text after it). */
static void geq_of(const orc_t *o, double T, double ux, double uy, double *geq) {
    double n[5];
    orc_neq_raw(T, ux, uy, o->c.sigma, o->c.varpi, n);
    matvec(5, o->MTinv, n, geq);
}

/* Buoyancy and external acceleration G = -g beta (T - T0) + a with gravity
 * along -y (Eq. 4 and the Boussinesq statement after it). */
static void body_G(const orc_cfg *c, double T, double ay, double *Gx, double *Gy) {
    *Gx = c->ax;
    *Gy = ay + c->gbeta * (T - c->T0);
}

/* Total force of Eq. 4 for a given velocity. */
static void force_of(const orc_cfg *c, double ux, double uy, double phi, double Gx, double Gy, double *Fx,
                     double *Fy) {
    double Fphi = c->forchheimer ? orc_ergun_Fphi(phi) : 0.0;
    double um = sqrt(ux * ux + uy * uy);
    *Fx = -phi * c->nu / c->K * ux - phi * Fphi / sqrt(c->K) * um * ux + phi * Gx;
    *Fy = -phi * c->nu / c->K * uy - phi * Fphi / sqrt(c->K) * um * uy + phi * Gy;
}

/* Macroscopic velocity by the explicit solution of Eqs. 22-23. */
static void velocity_of(const orc_cfg *c, double rho, double jx, double jy, double phi, double Gx, double Gy,
                        double *ux, double *uy) {
    double Fphi = c->forchheimer ? orc_ergun_Fphi(phi) : 0.0;
    double vx = jx / rho + 0.5 * phi * Gx;
    double vy = jy / rho + 0.5 * phi * Gy;
    double l0 = 0.5 * (1.0 + phi * 0.5 * c->nu / c->K);
    double l1 = phi * 0.5 * Fphi / sqrt(c->K);
    double vm = sqrt(vx * vx + vy * vy);
    double den = l0 + sqrt(l0 * l0 + l1 * vm);
    *ux = vx / den;
    *uy = vy / den;
}

/* Exposed for the pin tests: u and F from (rho, j, T) at one node. */
void orc_point_velocity(const orc_cfg *c, double rho, double jx, double jy, double T, double phi, double ay,
                        double *out /* ux, uy, Fx, Fy */) {
    double Gx, Gy;
    body_G(c, T, ay, &Gx, &Gy);
    velocity_of(c, rho, jx, jy, phi, Gx, Gy, &out[0], &out[1]);
    force_of(c, out[0], out[1], phi, Gx, Gy, &out[2], &out[3]);
}

/* Macroscopic state of an interior node from its pre-collision f, g:
 * Eq. 20 (rho), Eq. 36 (T), Eqs. 22-23 (u), Eq. 4 (F). */
static void interior_macros(const orc_t *o, int x, int y, double *rho, double *ux, double *uy, double *T) {
    const orc_cfg *c = &o->c;
    size_t n = (size_t)y * c->nx + x;
    const double *f = o->f + 9 * n, *g = o->g + 5 * n;
    double r = 0.0, jx = 0.0, jy = 0.0, st = 0.0;
    for (int i = 0; i < 9; ++i) {
        r += f[i];
        jx += EX9[i] * f[i];
        jy += EY9[i] * f[i];
    }
    for (int i = 0; i < 5; ++i) st += g[i];
    double t = st / c->sigma;
    double Gx, Gy;
    body_G(c, t, o->ay[y], &Gx, &Gy);
    velocity_of(c, r, jx, jy, o->phi[n], Gx, Gy, ux, uy);
    *rho = r;
    *T = t;
}

/* Flow collision of Eq. 11 at one node, f* = M^-1 N^-1 m~* (text after Eq. 18). */
void orc_collide_flow_ex(const double *M, const double *Minv, const double *Lam, int shift, const double *f,
                         double rho, double ux, double uy, double Fx, double Fy, double phi, double *fout) {
    double m[9], mt[9], meq[9], S[9], N[81], Ni[81], d[9], Ld[9], IS[9], ms[9], r[9];
    double IL[81];
    matvec(9, M, f, m);                                   /* Eq. 12 right */
    if (shift) {
        orc_matrix_N(ux, uy, phi, N);
        matvec(9, N, m, mt);                              /* Eq. 12 left */
        orc_meq_central(rho, meq);                        /* Eq. 16 */
        orc_S_central(rho, Fx, Fy, S);                    /* Eq. 17 */
        orc_matrix_Ninv(ux, uy, phi, Ni);                 /* Eq. A1 */
    } else {
        for (int i = 0; i < 9; ++i) mt[i] = m[i];         /* N = I (Sec. 2 end) */
        orc_meq_raw(rho, ux, uy, phi, meq);               /* Eq. 19 */
        orc_S_raw(rho, ux, uy, Fx, Fy, phi, S);
        for (int k = 0; k < 81; ++k) Ni[k] = (k % 10 == 0) ? 1.0 : 0.0;
    }
    for (int k = 0; k < 81; ++k) IL[k] = ((k % 10 == 0) ? 1.0 : 0.0) - 0.5 * Lam[k];
    for (int i = 0; i < 9; ++i) d[i] = mt[i] - meq[i];
    matvec(9, Lam, d, Ld);
    matvec(9, IL, S, IS);
    for (int i = 0; i < 9; ++i) ms[i] = mt[i] - Ld[i] + IS[i];   /* Eq. 11 */
    matvec(9, Ni, ms, r);
    matvec(9, Minv, r, fout);
}

/* Thermal collision of Eq. 28 at one node, g* = M_T^-1 N_T^-1 n~* (text after Eq. 35). */
void orc_collide_thermal_ex(const double *MT, const double *MTinv, const double *Q, int shift, const double *g,
                            double T, double ux, double uy, double sigma, double varpi, double *gout) {
    double n[5], nt[5], neq[5], N[25], Ni[25], d[5], Qd[5], ns[5], r[5];
    matvec(5, MT, g, n);
    if (shift) {
        orc_matrix_NT(ux, uy, sigma, N);
        matvec(5, N, n, nt);
        orc_neq_central(T, sigma, varpi, neq);            /* Eq. 32 */
        orc_matrix_NTinv(ux, uy, sigma, Ni);
    } else {
        for (int i = 0; i < 5; ++i) nt[i] = n[i];
        orc_neq_raw(T, ux, uy, sigma, varpi, neq);        /* Eq. 33 */
        for (int k = 0; k < 25; ++k) Ni[k] = (k % 6 == 0) ? 1.0 : 0.0;
    }
    for (int i = 0; i < 5; ++i) d[i] = nt[i] - neq[i];
    matvec(5, Q, d, Qd);
    for (int i = 0; i < 5; ++i) ns[i] = nt[i] - Qd[i];    /* Eq. 28 */
    matvec(5, Ni, ns, r);
    matvec(5, MTinv, r, gout);
}

/* Non-equilibrium extrapolation at wall node (x, y); see header comment. */
static void nee_node(orc_t *o, int x, int y) {
    const orc_cfg *c = &o->c;
    int nx = c->nx;
    int dx = 0, dy = 0, vert = -1, horz = -1;
    if (c->kind[0] && x == 0) { dx = 1; vert = 0; }
    if (c->kind[1] && x == nx - 1) { dx = -1; vert = 1; }
    if (c->kind[2] && y == 0) { dy = 1; horz = 2; }
    if (c->kind[3] && y == c->ny - 1) { dy = -1; horz = 3; }
    int side_u = vert >= 0 ? vert : horz;
    int side_t = -1;
    if (vert >= 0 && c->tdir[vert]) side_t = vert;
    else if (horz >= 0 && c->tdir[horz]) side_t = horz;
    int xf = x + dx, yf = y + dy, xff = x + 2 * dx, yff = y + 2 * dy;
    size_t nb = (size_t)y * nx + x, nf = (size_t)yf * nx + xf, nff = (size_t)yff * nx + xff;

    double rf, uxf, uyf, Tf;
    interior_macros(o, xf, yf, &rf, &uxf, &uyf, &Tf);
    double Tff = 0.0;
    for (int i = 0; i < 5; ++i) Tff += o->g[5 * nff + i];
    Tff /= c->sigma;
    double uw = c->uw[side_u], vw = c->vw[side_u];
    double Tb = side_t >= 0 ? c->Tw[side_t] : (4.0 * Tf - Tff) / 3.0;

    double fe_b[9], fe_f[9], ge_b[5], ge_f[5];
    feq_of(o, rf, uw, vw, o->phi[nb], fe_b);
    feq_of(o, rf, uxf, uyf, o->phi[nf], fe_f);
    geq_of(o, Tb, uw, vw, ge_b);
    geq_of(o, Tf, uxf, uyf, ge_f);
    for (int i = 0; i < 9; ++i) o->f[9 * nb + i] = fe_b[i] + (o->f[9 * nf + i] - fe_f[i]);
    for (int i = 0; i < 5; ++i) o->g[5 * nb + i] = ge_b[i] + (o->g[5 * nf + i] - ge_f[i]);
    o->wrho[nb] = rf;
    o->wux[nb] = uw;
    o->wuy[nb] = vw;
    o->wT[nb] = Tb;
}

static void apply_walls(orc_t *o) {
    const orc_cfg *c = &o->c;
    /* Wall nodes read only interior nodes, so the order does not matter. */
#pragma omp parallel for num_threads(c->nthreads) schedule(static)
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x)
            if (o->wall[(size_t)y * c->nx + x]) nee_node(o, x, y);
}

/* Macroscopic state of any node (walls: imposed values). */
static void node_macros(const orc_t *o, int x, int y, double *rho, double *ux, double *uy, double *T) {
    size_t n = (size_t)y * o->c.nx + x;
    if (o->wall[n]) {
        *rho = o->wrho[n]; *ux = o->wux[n]; *uy = o->wuy[n]; *T = o->wT[n];
    } else {
        interior_macros(o, x, y, rho, ux, uy, T);
    }
}

/* ---------------------------------------------------------------- public */
void *orc_create(const orc_cfg *cfg, const double *phi, const double *ay) {
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    if (!o) return NULL;
    o->c = *cfg;
    if (o->c.nthreads < 1) o->c.nthreads = 1;
    size_t n = (size_t)cfg->nx * cfg->ny;
    o->phi = (double *)malloc(n * sizeof(double));
    o->ay = (double *)malloc((size_t)cfg->ny * sizeof(double));
    o->f = (double *)calloc(9 * n, sizeof(double));
    o->g = (double *)calloc(5 * n, sizeof(double));
    o->fs = (double *)calloc(9 * n, sizeof(double));
    o->gs = (double *)calloc(5 * n, sizeof(double));
    o->wall = (unsigned char *)calloc(n, 1);
    o->wrho = (double *)calloc(n, sizeof(double));
    o->wux = (double *)calloc(n, sizeof(double));
    o->wuy = (double *)calloc(n, sizeof(double));
    o->wT = (double *)calloc(n, sizeof(double));
    if (!o->phi || !o->ay || !o->f || !o->g || !o->fs || !o->gs || !o->wall || !o->wrho || !o->wux || !o->wuy ||
        !o->wT)
        return NULL;
    memcpy(o->phi, phi, n * sizeof(double));
    memcpy(o->ay, ay, (size_t)cfg->ny * sizeof(double));
    orc_matrix_M(o->M);
    orc_invert(9, o->M, o->Minv);
    orc_matrix_MT(o->MT);
    orc_invert(5, o->MT, o->MTinv);
    orc_matrix_Lambda(cfg->s0, cfg->s1, cfg->sb, cfg->sv, cfg->s3, cfg->s4, o->L);
    for (int k = 0; k < 25; ++k) o->Q[k] = 0.0;
    o->Q[0] = cfg->zT; o->Q[6] = cfg->za; o->Q[12] = cfg->za; o->Q[18] = cfg->ze; o->Q[24] = cfg->zn;
    for (int y = 0; y < cfg->ny; ++y)
        for (int x = 0; x < cfg->nx; ++x) o->wall[(size_t)y * cfg->nx + x] = (unsigned char)is_wall_node(cfg, x, y);
    return o;
}

void orc_destroy(void *h) {
    orc_t *o = (orc_t *)h;
    if (!o) return;
    free(o->phi); free(o->ay); free(o->f); free(o->g); free(o->fs); free(o->gs);
    free(o->wall); free(o->wrho); free(o->wux); free(o->wuy); free(o->wT);
    free(o);
}

/* Start from equilibrium: f = f^eq(rho, u; phi), g = g^eq(T, u) per node,
 * then reconstruct the wall nodes. */
void orc_set_fields(void *h, const double *rho, const double *ux, const double *uy, const double *T) {
    orc_t *o = (orc_t *)h;
    const orc_cfg *c = &o->c;
    size_t n = (size_t)c->nx * c->ny;
    for (size_t k = 0; k < n; ++k) {
        feq_of(o, rho[k], ux[k], uy[k], o->phi[k], o->f + 9 * k);
        geq_of(o, T[k], ux[k], uy[k], o->g + 5 * k);
    }
    apply_walls(o);
}

/* Advance nsteps time steps: collide every node, stream, rebuild walls. */
void orc_step(void *h, int64_t nsteps) {
    orc_t *o = (orc_t *)h;
    const orc_cfg *c = &o->c;
    int nx = c->nx, ny = c->ny;
    for (int64_t s = 0; s < nsteps; ++s) {
#pragma omp parallel for num_threads(c->nthreads) schedule(static)
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                size_t n = (size_t)y * nx + x;
                double rho, ux, uy, T, Gx, Gy, Fx, Fy;
                node_macros(o, x, y, &rho, &ux, &uy, &T);
                body_G(c, T, o->ay[y], &Gx, &Gy);
                force_of(c, ux, uy, o->phi[n], Gx, Gy, &Fx, &Fy);
                orc_collide_flow_ex(o->M, o->Minv, o->L, c->shift, o->f + 9 * n, rho, ux, uy, Fx, Fy, o->phi[n],
                                    o->fs + 9 * n);
                orc_collide_thermal_ex(o->MT, o->MTinv, o->Q, c->shift, o->g + 5 * n, T, ux, uy, c->sigma, c->varpi,
                                       o->gs + 5 * n);
            }
        }
        /* Streaming, Eq. 18 and Eq. 35: push each post-collision value to the
         * neighbour along e_i; periodic sides wrap, wall sides drop it. */
#pragma omp parallel for num_threads(c->nthreads) schedule(static)
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                size_t n = (size_t)y * nx + x;
                for (int i = 0; i < 9; ++i) {
                    int xt = x + EX9[i], yt = y + EY9[i];
                    if (xt < 0 || xt >= nx) { if (c->kind[0]) continue; xt = (xt + nx) % nx; }
                    if (yt < 0 || yt >= ny) { if (c->kind[2]) continue; yt = (yt + ny) % ny; }
                    size_t t = (size_t)yt * nx + xt;
                    o->f[9 * t + i] = o->fs[9 * n + i];
                    if (i < 5) o->g[5 * t + i] = o->gs[5 * n + i];
                }
            }
        }
        apply_walls(o);
    }
}

/* Macroscopic fields at the current time level (any pointer may be NULL). */
void orc_macros(void *h, double *rho, double *ux, double *uy, double *T) {
    orc_t *o = (orc_t *)h;
    const orc_cfg *c = &o->c;
#pragma omp parallel for num_threads(c->nthreads) schedule(static)
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            size_t n = (size_t)y * c->nx + x;
            double r, a, b, t;
            node_macros(o, x, y, &r, &a, &b, &t);
            if (rho) rho[n] = r;
            if (ux) ux[n] = a;
            if (uy) uy[n] = b;
            if (T) T[n] = t;
        }
}

/* Raw pre-collision distributions (9*nx*ny and 5*nx*ny, node-major). */
void orc_get_state(void *h, double *f, double *g) {
    orc_t *o = (orc_t *)h;
    size_t n = (size_t)o->c.nx * o->c.ny;
    if (f) memcpy(f, o->f, 9 * n * sizeof(double));
    if (g) memcpy(g, o->g, 5 * n * sizeof(double));
}

void orc_set_state(void *h, const double *f, const double *g) {
    orc_t *o = (orc_t *)h;
    size_t n = (size_t)o->c.nx * o->c.ny;
    if (f) memcpy(o->f, f, 9 * n * sizeof(double));
    if (g) memcpy(o->g, g, 5 * n * sizeof(double));
    apply_walls(o);
}

/* Single-node helpers for the pin tests (standard matrices built inside). */
void orc_feq(double rho, double ux, double uy, double phi, double *out) {
    double M[81], Mi[81], m[9];
    orc_matrix_M(M);
    orc_invert(9, M, Mi);
    orc_meq_raw(rho, ux, uy, phi, m);
    matvec(9, Mi, m, out);
}

void orc_geq(double T, double ux, double uy, double sigma, double varpi, double *out) {
    double M[25], Mi[25], n[5];
    orc_matrix_MT(M);
    orc_invert(5, M, Mi);
    orc_neq_raw(T, ux, uy, sigma, varpi, n);
    matvec(5, Mi, n, out);
}

void orc_collide_flow(const double *f, double rho, double ux, double uy, double Fx, double Fy, double phi,
                      double s0, double s1, double sb, double sv, double s3, double s4, int shift, double *out) {
    double M[81], Mi[81], L[81];
    orc_matrix_M(M);
    orc_invert(9, M, Mi);
    orc_matrix_Lambda(s0, s1, sb, sv, s3, s4, L);
    orc_collide_flow_ex(M, Mi, L, shift, f, rho, ux, uy, Fx, Fy, phi, out);
}

void orc_collide_thermal(const double *g, double T, double ux, double uy, double sigma, double varpi, double zT,
                         double za, double ze, double zn, int shift, double *out) {
    double M[25], Mi[25], Q[25];
    orc_matrix_MT(M);
    orc_invert(5, M, Mi);
    for (int k = 0; k < 25; ++k) Q[k] = 0.0;
    Q[0] = zT; Q[6] = za; Q[12] = za; Q[18] = ze; Q[24] = zn;
    orc_collide_thermal_ex(M, Mi, Q, shift, g, T, ux, uy, sigma, varpi, out);
}

int orc_sizeof_cfg(void) { return (int)sizeof(orc_cfg); }
