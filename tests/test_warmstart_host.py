"""Host-side pieces of the learned warm start: the centro-symmetry of the
heated cavity behind the training-set augmentation (checked on the oracle),
the feature and target maps and the velocity-scale fit.  No GPU."""
import math

import numpy as np

from paper_2110_05943_gb300 import surrogate
from paper_2110_05943_gb300.inputs import gaussian_random_field, warmstart_cases


def _R(z):
    return z[::-1, ::-1]


def test_rotated_porosity_gives_the_rotated_solution(orc):
    """A cavity heated from the west and cooled from the east, run on eps(x)
    and on eps(R x): the second run reproduces (-u, 1 - T, rho)(R x) of the
    first up to the weak compressibility of the LB fluid (measured on 24^2,
    Ra 1e4: u 0.18 %, T 0.55 %, density deviation 0.6 %), which is what
    surrogate.augment_rot180 assumes."""
    n = 24
    phi = np.clip(0.6 + 0.1 * gaussian_random_field(n, n, 6.0, seed=5), 0.3, 0.95)
    p = orc.Problem(nx=n, ny=n, Ra=1e4, Da=1e-2, Pr=0.71)
    a = orc.Oracle(p, phi=phi, nthreads=4)
    b = orc.Oracle(p, phi=np.ascontiguousarray(_R(phi)), nthreads=4)
    a.step(4000)
    b.step(4000)
    ra, uxa, uya, Ta = a.macros()
    rb, uxb, uyb, Tb = b.macros()
    um = np.hypot(uxa, uya).max()
    assert np.abs(uxb + _R(uxa)).max() < 5e-3 * um
    assert np.abs(uyb + _R(uya)).max() < 5e-3 * um
    assert np.abs(Tb - (1.0 - _R(Ta))).max() < 1e-2
    da, db = ra - ra.mean(), rb - rb.mean()
    assert np.abs(db - _R(da)).max() < 3e-2 * np.abs(da).max()        # symmetric ...
    assert np.abs(db + _R(da)).max() > 1.0 * np.abs(da).max()         # ... not antisymmetric

    # the augmentation maps the first run's (features, targets) onto the second's
    vs = 0.01
    Xa = surrogate.features(phi, 1e4, 1e-2, 0.71, 1.0)[None]
    Xb = surrogate.features(_R(phi), 1e4, 1e-2, 0.71, 1.0)[None]
    Ya = surrogate.targets(ra, uxa, uya, Ta, vs)[None]
    Yb = surrogate.targets(rb, uxb, uyb, Tb, vs)[None]
    Xr, Yr = surrogate.augment_rot180(Xa, Ya)
    assert np.array_equal(Xr, Xb)
    scale = np.abs(Yb).max(axis=(0, 1, 2))
    assert np.all(np.abs(Yr - Yb).max(axis=(0, 1, 2)) < 3e-2 * scale)
    X2, Y2 = surrogate.augment_rot180(Xr, Yr)                          # an involution
    assert np.array_equal(X2, Xa) and np.array_equal(Y2, Ya)


def test_targets_and_fields_are_inverse():
    rng = np.random.default_rng(0)
    h, w = 16, 20
    rho = 1.0 + 1e-3 * rng.standard_normal((h, w))
    ux, uy = 1e-3 * rng.standard_normal((2, h, w))
    T = rng.uniform(0, 1, (h, w))
    Y = surrogate.targets(rho, ux, uy, T, 2e-3)
    r2, u2, v2, T2 = surrogate.fields_from(Y, 2e-3)
    assert np.allclose(u2, ux, rtol=1e-6, atol=1e-12) and np.allclose(v2, uy, rtol=1e-6, atol=1e-12)
    assert np.allclose(T2, T, atol=1e-6)
    assert np.allclose(r2 - 1.0, rho - rho.mean(), atol=1e-8)          # mean density reset to 1
    Tc = surrogate.conduction_T(h, w)
    assert Tc[0, 0] == 1.0 and Tc[0, -1] == 0.0 and np.allclose(Tc[:, 1:] - Tc[:, :-1], -1.0 / (w - 1))


def test_velocity_scale_fit_recovers_a_power_law():
    """u_rms = u_c 0.3 Ra^0.4 Da^0.5 sigma^-0.2 is recovered exactly by the
    log-linear fit (it lies in the fitted family)."""
    rng = np.random.default_rng(1)
    prm = [(10 ** rng.uniform(3, 6), 10 ** rng.uniform(-4, -1), rng.uniform(0.7, 1.0), rng.uniform(0.5, 2),
            rng.uniform(0.4, 0.9)) for _ in range(50)]
    u = [surrogate.U_C * 0.3 * Ra ** 0.4 * Da ** 0.5 * sg ** -0.2 for Ra, Da, Pr, sg, e in prm]
    coef = surrogate.fit_velocity_scale(prm, u)
    for p, ui in zip(prm[:5], u[:5]):
        assert abs(surrogate.velocity_scale(coef, *p) / ui - 1) < 1e-9


def test_features_and_cases():
    cases = warmstart_cases(4, seed=11)
    c, phi = cases[0]
    assert phi.shape == (128, 128) and 0.3 <= phi.min() and phi.max() <= 0.95
    assert 1e3 <= c.Ra <= 1e6 and 1e-4 <= c.Da <= 1e-1 and 0.5 <= c.sigma <= 2 and 0.7 <= c.Pr <= 1.0
    X = surrogate.features(phi, c.Ra, c.Da, c.Pr, c.sigma)
    assert X.shape == (128, 128, surrogate.N_IN)
    assert np.all(X[..., 1] == X[0, 0, 1]) and abs(X[0, 0, 1] - (math.log10(c.Ra) - 4.5) / 0.87) < 1e-6
    assert X[0, 0, 5] == -0.5 and X[0, -1, 5] == 0.5 and X[0, 0, 6] == -0.5 and X[-1, 0, 6] == 0.5
    again = warmstart_cases(4, seed=11)
    assert all(np.array_equal(a[1], b[1]) and a[0] == b[0] for a, b in zip(cases, again))
