"""Pins of the CPU oracle's per-node algebra against what the paper and the
mathematics fix independently of the oracle's own formulas.

Each check compares two *different* statements of the method (e.g. the raw
equilibrium of Eq. 19 shifted by Eq. 14 against the central equilibrium of
Eq. 16), or the oracle against a brute-force definition (Eq. 8, Eq. 25), so
that a dropped term, a wrong sign or index, or a transposed operand in any
one of them fails a test.
"""
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)
MOM9 = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (2, 1), (1, 2), (2, 2)]
MOM5 = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2)]


def _load(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#")


def _central_T(ux, uy, nq, moms):
    """Brute-force central-moment transform of Eq. 8 / Eq. 25:
    row (m, n) = (e_x - u_x)^m (e_y - u_y)^n."""
    return np.array([[(EX[i] - ux) ** m * (EY[i] - uy) ** n for i in range(nq)] for (m, n) in moms])


def _rng(seed=1):
    return np.random.default_rng(seed)


# ------------------------------------------------------------------ matrices
def test_M_matches_printed_eq13(orc):
    assert np.array_equal(orc.mat("M"), _load("eq13_M.txt"))


def test_MT_matches_printed_eq30(orc):
    assert np.array_equal(orc.mat("MT"), _load("eq30_MT.txt"))


def test_numeric_inverses(orc):
    M, MT = orc.mat("M"), orc.mat("MT")
    np.testing.assert_allclose(orc.invert(M) @ M, np.eye(9), atol=1e-15)
    np.testing.assert_allclose(orc.invert(M), np.linalg.inv(M), atol=1e-15)
    np.testing.assert_allclose(orc.invert(MT), np.linalg.inv(MT), atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_N_times_A1_is_identity(orc, seed):
    r = _rng(seed)
    ux, uy = r.uniform(-0.3, 0.3, 2)
    phi = r.uniform(0.2, 1.0)
    P = orc.mat("N", ux, uy, phi) @ orc.mat("Ninv", ux, uy, phi)
    np.testing.assert_allclose(P, np.eye(9), atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_NT_times_inverse_is_identity(orc, seed):
    r = _rng(seed)
    ux, uy = r.uniform(-0.3, 0.3, 2)
    sigma = r.uniform(0.3, 3.0)
    P = orc.mat("NT", ux, uy, sigma) @ orc.mat("NTinv", ux, uy, sigma)
    np.testing.assert_allclose(P, np.eye(5), atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_shift_at_phi1_equals_brute_force_central_moments(orc, seed):
    """phi = 1: N M f must be Eq. 8's central moments, summed directly."""
    r = _rng(seed)
    ux, uy = r.uniform(-0.2, 0.2, 2)
    f = r.uniform(0.0, 0.5, 9)
    got = orc.mat("N", ux, uy, 1.0) @ orc.mat("M") @ f
    want = _central_T(ux, uy, 9, MOM9) @ f
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_thermal_shift_at_sigma1_equals_brute_force(orc, seed):
    """sigma = 1: N_T M_T g must be Eq. 25's central moments when sum g = T."""
    r = _rng(seed)
    ux, uy = r.uniform(-0.2, 0.2, 2)
    g = r.uniform(0.0, 0.5, 5)
    got = orc.mat("NT", ux, uy, 1.0) @ orc.mat("MT") @ g
    want = _central_T(ux, uy, 5, MOM5) @ g
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


def test_porous_shift_differs_from_eq8_away_from_phi1(orc):
    """The porous N is not Eq. 8's shift when phi != 1 (it is the paper's
    modification); guards against the oracle silently ignoring phi."""
    f = np.linspace(0.05, 0.2, 9)
    ux, uy, phi = 0.1, -0.05, 0.6
    got = orc.mat("N", ux, uy, phi) @ orc.mat("M") @ f
    plain = _central_T(ux, uy, 9, MOM9) @ f
    assert np.max(np.abs(got - plain)) > 1e-4


# ------------------------------------------------------------ equilibria / forcing
@pytest.mark.parametrize("seed", range(6))
def test_shifted_raw_equilibrium_is_central_equilibrium(orc, seed):
    """Eq. 14 applied to Eq. 19's m^eq gives Eq. 16's central equilibrium."""
    r = _rng(seed)
    rho = r.uniform(0.8, 1.2)
    ux, uy = r.uniform(-0.2, 0.2, 2)
    phi = r.uniform(0.3, 1.0)
    got = orc.mat("N", ux, uy, phi) @ orc.vec("meq_raw", 9, rho, ux, uy, phi)
    want = orc.vec("meq_central", 9, rho)
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-16 * 16)


@pytest.mark.parametrize("seed", range(6))
def test_shifted_raw_forcing_is_central_forcing(orc, seed):
    """Eq. 14 applied to Eq. 19's S gives Eq. 17's central forcing."""
    r = _rng(seed)
    rho = r.uniform(0.8, 1.2)
    ux, uy, Fx, Fy = r.uniform(-0.2, 0.2, 4)
    phi = r.uniform(0.3, 1.0)
    got = orc.mat("N", ux, uy, phi) @ orc.vec("S_raw", 9, rho, ux, uy, Fx, Fy, phi)
    want = orc.vec("S_central", 9, rho, Fx, Fy)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_thermal_shift_of_raw_equilibrium(orc, seed):
    """Eq. 31 applied to Eq. 33 gives Eq. 32."""
    r = _rng(seed)
    T = r.uniform(-1, 2)
    ux, uy = r.uniform(-0.2, 0.2, 2)
    sigma = r.uniform(0.4, 2.5)
    got = orc.mat("NT", ux, uy, sigma) @ orc.vec("neq_raw", 5, T, ux, uy, sigma, 0.25)
    want = orc.vec("neq_central", 5, T, sigma, 0.25)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_geq_matches_explicit_eq34(orc, seed):
    """M_T^-1 n^eq (Eq. 33) equals the explicit distribution of Eq. 34."""
    r = _rng(seed)
    T = r.uniform(-1, 2)
    ux, uy = r.uniform(-0.2, 0.2, 2)
    sigma, w = r.uniform(0.4, 2.5), r.uniform(0.1, 0.9)
    g = orc.geq(T, ux, uy, sigma, w)
    u2 = ux * ux + uy * uy
    eq34 = np.array([
        sigma * T - w * T - u2 * T,
        w / 4 * T + 0.5 * ux * T + 0.5 * ux * ux * T,
        w / 4 * T + 0.5 * uy * T + 0.5 * uy * uy * T,
        w / 4 * T - 0.5 * ux * T + 0.5 * ux * ux * T,
        w / 4 * T - 0.5 * uy * T + 0.5 * uy * uy * T,
    ])
    np.testing.assert_allclose(g, eq34, rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_feq_velocity_moments(orc, seed):
    """f^eq = M^-1 m^eq has the moments its definition requires, summed
    directly over the nine velocities: density, momentum, and the porous
    second moments rho (c_s^2 delta + u u / phi) (Eq. 19)."""
    r = _rng(seed)
    rho = r.uniform(0.8, 1.2)
    ux, uy = r.uniform(-0.2, 0.2, 2)
    phi = r.uniform(0.3, 1.0)
    f = orc.feq(rho, ux, uy, phi)
    assert math.isclose(f.sum(), rho, rel_tol=0, abs_tol=1e-15)
    assert math.isclose((EX * f).sum(), rho * ux, abs_tol=1e-15)
    assert math.isclose((EY * f).sum(), rho * uy, abs_tol=1e-15)
    assert math.isclose((EX * EX * f).sum(), rho / 3 + rho * ux * ux / phi, abs_tol=1e-15)
    assert math.isclose((EY * EY * f).sum(), rho / 3 + rho * uy * uy / phi, abs_tol=1e-15)
    assert math.isclose((EX * EY * f).sum(), rho * ux * uy / phi, abs_tol=1e-15)


def test_rest_equilibrium_weights(orc):
    """At rest the D2Q9 equilibrium is rho (16, 4, 4, 4, 4, 1, 1, 1, 1)/36 (the
    textbook D2Q9 weights) and the D2Q5 one is ((sigma - varpi) T, varpi T / 4, ...)."""
    f = orc.feq(1.3, 0.0, 0.0, 0.5)
    np.testing.assert_allclose(f, 1.3 * np.array([16, 4, 4, 4, 4, 1, 1, 1, 1]) / 36, atol=1e-16)
    g = orc.geq(0.7, 0.0, 0.0, 1.5, 0.25)
    np.testing.assert_allclose(g, [(1.5 - 0.25) * 0.7] + [0.25 * 0.7 / 4] * 4, atol=1e-16)


def test_ergun_inertia_coefficient(orc):
    """Eq. 5: F_phi = 1.75 / sqrt(150 phi^3); F_phi(1) = 1.75/sqrt(150) ~ 0.1429."""
    assert math.isclose(orc.ergun_Fphi(1.0), 0.14288690166235207, rel_tol=1e-14)
    # F_phi scales as phi^(-3/2)
    assert math.isclose(orc.ergun_Fphi(0.25) / orc.ergun_Fphi(1.0), 8.0, rel_tol=1e-14)


# ------------------------------------------------------------ implicit velocity
def _cfg(orc, forchheimer=True, K=2.5, nu=0.05, gbeta=1e-3, T0=0.5, ax=1e-4):
    c = orc._Cfg()
    c.nu, c.nu_e, c.K, c.gbeta, c.T0, c.ax = nu, nu, K, gbeta, T0, ax
    c.forchheimer = int(forchheimer)
    return c


@pytest.mark.parametrize("forch", [True, False])
@pytest.mark.parametrize("seed", range(4))
def test_implicit_velocity_solves_eq21(orc, forch, seed):
    """Eqs. 22-23 give the u that satisfies rho u = sum e f + rho F(u)/2 with
    F from Eq. 4 -- checked by substituting back into Eq. 21."""
    import ctypes
    r = _rng(seed)
    c = _cfg(orc, forch, K=r.uniform(0.5, 50), nu=r.uniform(0.01, 0.2))
    rho = r.uniform(0.9, 1.1)
    jx, jy = r.uniform(-0.1, 0.1, 2)
    T, phi, ay = r.uniform(0, 1), r.uniform(0.3, 1.0), r.uniform(-1e-3, 1e-3)
    out = np.zeros(4)
    orc.lib().orc_point_velocity(ctypes.byref(c), rho, jx, jy, T, phi, ay, orc._p(out))
    ux, uy, Fx, Fy = out
    # F re-derived from Eq. 4 at the returned u
    Fphi = 1.75 / math.sqrt(150 * phi ** 3) if forch else 0.0
    um = math.hypot(ux, uy)
    Gx, Gy = c.ax, ay + c.gbeta * (T - c.T0)
    Fx2 = -phi * c.nu / c.K * ux - phi * Fphi / math.sqrt(c.K) * um * ux + phi * Gx
    Fy2 = -phi * c.nu / c.K * uy - phi * Fphi / math.sqrt(c.K) * um * uy + phi * Gy
    assert math.isclose(Fx, Fx2, rel_tol=1e-13, abs_tol=1e-18)
    assert math.isclose(rho * ux, jx + 0.5 * rho * Fx2, rel_tol=1e-13, abs_tol=1e-17)
    assert math.isclose(rho * uy, jy + 0.5 * rho * Fy2, rel_tol=1e-13, abs_tol=1e-17)


# ------------------------------------------------------------ collision
def _random_node(r):
    rho = r.uniform(0.9, 1.1)
    ux, uy = r.uniform(-0.1, 0.1, 2)
    phi = r.uniform(0.3, 1.0)
    return rho, ux, uy, phi


@pytest.mark.parametrize("seed", range(5))
def test_collision_conserves_mass_and_sets_first_central_moment(orc, seed):
    """sum f* = rho (s_0 acts on a conserved moment) and the post-collision
    central moment k~10* equals rho F_x / 2 for any s_1 (Eq. 11 with Eq. 17),
    provided u satisfies Eq. 21."""
    r = _rng(seed)
    rho, ux, uy, phi = _random_node(r)
    Fx, Fy = r.uniform(-1e-3, 1e-3, 2)
    f = orc.feq(rho, ux, uy, phi) + r.uniform(-1e-3, 1e-3, 9)
    # make u consistent with Eq. 21: rho u = sum e f + rho F / 2
    f0 = f.copy()
    jx, jy = (EX * f0).sum(), (EY * f0).sum()
    rho = f0.sum()
    ux, uy = (jx + 0.5 * rho * Fx) / rho, (jy + 0.5 * rho * Fy) / rho
    for s1 in (1.0, 0.7, 1.6):
        fs = orc.collide_flow(f0, rho, ux, uy, Fx, Fy, phi, sv=1.3, s1=s1)
        assert math.isclose(fs.sum(), rho, rel_tol=0, abs_tol=1e-15)
        mt = orc.mat("N", ux, uy, phi) @ orc.mat("M") @ fs
        assert math.isclose(mt[1], 0.5 * rho * Fx, abs_tol=1e-16)
        assert math.isclose(mt[2], 0.5 * rho * Fy, abs_tol=1e-16)


@pytest.mark.parametrize("shift", [True, False])
def test_rest_state_is_fixed_point(orc, shift):
    f = orc.feq(1.0, 0.0, 0.0, 0.6)
    fs = orc.collide_flow(f, 1.0, 0.0, 0.0, 0.0, 0.0, 0.6, sv=1.7, shift=shift)
    np.testing.assert_allclose(fs, f, atol=1e-16)
    g = orc.geq(0.3, 0.0, 0.0, 1.4)
    gs = orc.collide_thermal(g, 0.3, 0.0, 0.0, 1.4, za=1.2, shift=shift)
    np.testing.assert_allclose(gs, g, atol=1e-16)


@pytest.mark.parametrize("seed", range(4))
def test_equilibrium_with_velocity_is_fixed_point(orc, seed):
    """Without force, f^eq(rho, u; phi) is invariant under the collision
    (the shifted equilibrium is exactly Eq. 16); same for g^eq and Eq. 32."""
    r = _rng(seed)
    rho, ux, uy, phi = _random_node(r)
    f = orc.feq(rho, ux, uy, phi)
    np.testing.assert_allclose(orc.collide_flow(f, rho, ux, uy, 0, 0, phi, sv=1.5), f, atol=1e-15)
    sigma = r.uniform(0.5, 2.0)
    g = orc.geq(0.4, ux, uy, sigma)
    np.testing.assert_allclose(orc.collide_thermal(g, 0.4, ux, uy, sigma, za=1.3), g, atol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_thermal_collision_conserves_energy(orc, seed):
    r = _rng(seed)
    ux, uy = r.uniform(-0.1, 0.1, 2)
    sigma = r.uniform(0.5, 2.0)
    g = orc.geq(0.6, ux, uy, sigma) + r.uniform(-1e-3, 1e-3, 5)
    T = g.sum() / sigma
    gs = orc.collide_thermal(g, T, ux, uy, sigma, za=1.4)
    assert math.isclose(gs.sum(), g.sum(), rel_tol=0, abs_tol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_phi1_collision_equals_plain_central_moment_clb(orc, seed):
    """phi -> 1 reduces the method to the CLB of Fei et al. (end of Sec. 2):
    transform with the brute-force (e - u) moments of Eq. 8, relax every
    central moment towards Eq. 16 with Eq. 17's forcing, transform back by
    a numeric inverse of that brute-force matrix."""
    r = _rng(seed)
    rho, ux, uy, _ = _random_node(r)
    Fx, Fy = r.uniform(-1e-3, 1e-3, 2)
    f = orc.feq(rho, ux, uy, 1.0) + r.uniform(-1e-3, 1e-3, 9)
    sv, s3, s4 = 1.45, 1.2, 1.8
    Tm = _central_T(ux, uy, 9, MOM9)
    k = Tm @ f
    cs2 = 1 / 3
    keq = np.array([rho, 0, 0, rho * cs2, rho * cs2, 0, 0, 0, rho * cs2 * cs2])
    S = np.array([0, rho * Fx, rho * Fy, 0, 0, 0, cs2 * rho * Fy, cs2 * rho * Fx, 0])
    rates = np.array([1, 1, 1, sv, sv, sv, s3, s3, s4])
    kstar = k - rates * (k - keq) + (1 - rates / 2) * S
    want = np.linalg.solve(Tm, kstar)
    got = orc.collide_flow(f, rho, ux, uy, Fx, Fy, 1.0, sv=sv, s3=s3, s4=s4)
    np.testing.assert_allclose(got, want, rtol=0, atol=5e-15)


def test_unit_shift_is_raw_moment_mrt(orc):
    """N = N_T = I (end of Sec. 2): collision in raw moments towards Eq. 19's
    m^eq with Eq. 19's S; checked against a direct raw-moment relaxation."""
    r = _rng(11)
    rho, ux, uy, phi = _random_node(r)
    Fx, Fy = 2e-4, -3e-4
    f = orc.feq(rho, ux, uy, phi) + r.uniform(-1e-3, 1e-3, 9)
    M = orc.mat("M")
    m = M @ f
    meq = orc.vec("meq_raw", 9, rho, ux, uy, phi)
    S = orc.vec("S_raw", 9, rho, ux, uy, Fx, Fy, phi)
    rates = np.array([1, 1, 1, 1.3, 1.3, 1.3, 1.2, 1.2, 1.8])
    want = np.linalg.solve(M, m - rates * (m - meq) + (1 - rates / 2) * S)
    got = orc.collide_flow(f, rho, ux, uy, Fx, Fy, phi, sv=1.3, shift=False)
    np.testing.assert_allclose(got, want, rtol=0, atol=5e-15)


def test_lambda_block_couples_normal_moments(orc):
    """Eq. 15: the (k20, k02) block is [[s+, s-], [s-, s+]]."""
    L = orc.mat("Lambda", 1.0, 1.0, 1.6, 1.2, 1.3, 1.7)
    assert L[3, 3] == pytest.approx(1.4) and L[4, 4] == pytest.approx(1.4)
    assert L[3, 4] == pytest.approx(0.2) and L[4, 3] == pytest.approx(0.2)
    assert L[5, 5] == 1.2 and L[6, 6] == 1.3 and L[7, 7] == 1.3 and L[8, 8] == 1.7


# ------------------------------------------------------------ parameter mapping
def test_eq46_mapping_consistent_with_characteristic_velocity(orc):
    """Eq. 46 with Ma = u_c / c_s and u_c = sqrt(g beta dT L) must reproduce
    g beta dT L = (Ma c_s)^2 through the Rayleigh number of Eq. 38."""
    p = orc.Problem(nx=64, ny=64, Ra=1e5, Da=1e-3, Pr=0.71, J=1.0)
    lat = orc.lattice_params(p)
    uc2 = (0.1 / math.sqrt(3)) ** 2
    assert math.isclose(lat.gbeta * lat.L, uc2, rel_tol=1e-13)
    assert math.isclose(lat.nu / lat.alpha, 0.71, rel_tol=1e-13)
    assert math.isclose(lat.K, 1e-3 * 63 ** 2, rel_tol=1e-15)
    # Eq. 46 second part = Eq. 37 with alpha_e = Gamma alpha
    assert math.isclose(lat.alpha_e, lat.alpha, rel_tol=1e-13)
