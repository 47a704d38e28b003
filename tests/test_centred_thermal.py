"""The rest-centred thermal arithmetic of the FP16 forms rests on two exact
identities; both are checked here against the oracle's independent D2Q5
collision and equilibrium (Eqs. 28-36), on the CPU.

With q_i(u) = g^eq_i(1, u), the rest state g_rest = T0 q(0), g~ = g - g_rest
and T~ = T - T0:
  (1) g^eq_i(T, u) - T0 q_i(0) = T~ (sigma - 2 cT2) - T |u|^2       (i = 0)
                              = (T~ cT2 + T u_d (u_d +- 1)) / 2      (i = 1..4)
  (2) collide(g~ + g_rest, T~ + T0) - g_rest = collide(g~, T~) + T0 k(u),
      k_0 = -b |u|^2, k_{1,3} = (b X^2 +- a X) / 2, k_{2,4} = (b Y^2 +- a Y) / 2,
      a = zeta_a, b = 1 - 2 (1 - zeta_a) with the shift, b = 1 without,
for the relaxation rates the method uses (zeta_T = zeta_e = zeta_nu = 1)."""
import numpy as np
import pytest


def _centred_geq(Tt, X, Y, sigma, varpi, T0):
    cT2 = 0.5 * varpi
    T = Tt + T0
    return np.array([Tt * (sigma - 2 * cT2) - T * (X * X + Y * Y),
                     0.5 * (Tt * cT2 + T * X * (X + 1)),
                     0.5 * (Tt * cT2 + T * Y * (Y + 1)),
                     0.5 * (Tt * cT2 + T * X * (X - 1)),
                     0.5 * (Tt * cT2 + T * Y * (Y - 1))])


def _k(X, Y, za, shift):
    a = za
    b = 1.0 - 2.0 * (1.0 - za) if shift else 1.0
    return np.array([-b * (X * X + Y * Y), 0.5 * (b * X * X + a * X), 0.5 * (b * Y * Y + a * Y),
                     0.5 * (b * X * X - a * X), 0.5 * (b * Y * Y - a * Y)])


def test_centred_equilibrium_identity(orc):
    rng = np.random.default_rng(3)
    for _ in range(20):
        T0, Tt = rng.uniform(-1, 1), rng.uniform(-0.5, 0.5)
        X, Y = rng.uniform(-0.1, 0.1, 2)
        sigma, varpi = rng.uniform(0.5, 2.0), rng.uniform(0.1, 0.5)
        want = orc.geq(Tt + T0, X, Y, sigma, varpi) - orc.geq(T0, 0.0, 0.0, sigma, varpi)
        assert np.allclose(_centred_geq(Tt, X, Y, sigma, varpi, T0), want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("shift", [True, False])
def test_centred_collision_identity(orc, shift):
    rng = np.random.default_rng(4)
    for _ in range(20):
        T0 = rng.uniform(-1, 1)
        X, Y = rng.uniform(-0.1, 0.1, 2)
        sigma, varpi, za = rng.uniform(0.5, 2.0), rng.uniform(0.1, 0.5), rng.uniform(0.3, 1.9)
        gt = rng.uniform(-0.05, 0.05, 5)
        Tt = gt.sum() / sigma
        g_rest = orc.geq(T0, 0.0, 0.0, sigma, varpi)
        lhs = orc.collide_thermal(gt + g_rest, Tt + T0, X, Y, sigma, za, varpi, shift=shift) - g_rest
        rhs = orc.collide_thermal(gt, Tt, X, Y, sigma, za, varpi, shift=shift) + T0 * _k(X, Y, za, shift)
        assert np.allclose(lhs, rhs, rtol=0, atol=1e-14), (lhs, rhs)


def test_a_dropped_correction_term_is_detected(orc):
    """Without the T0 k(u) term the identity fails by O(T0 |u|): the check
    above is sensitive to the correction it pins."""
    T0, X, Y, sigma, varpi, za = 0.5, 0.03, -0.02, 1.0, 0.25, 1.2
    gt = np.array([0.01, -0.004, 0.003, 0.002, -0.001])
    Tt = gt.sum() / sigma
    g_rest = orc.geq(T0, 0.0, 0.0, sigma, varpi)
    lhs = orc.collide_thermal(gt + g_rest, Tt + T0, X, Y, sigma, za, varpi) - g_rest
    rhs = orc.collide_thermal(gt, Tt, X, Y, sigma, za, varpi)
    assert np.abs(lhs - rhs).max() > 1e-3
