"""Physics checks of the CUDA path at sizes the oracle cannot reach in a
test: Table 1 of the paper, the sigma-invariance of the steady Nusselt
number (Sec. 3.2) and the closed-form Brinkman channel of the 1024 x 256
porous-channel workload."""
import math
import os

import numpy as np
import pytest

from cases import CHANNEL_X, build

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def steady(sim, chunk=2000, tol=1e-10, max_steps=3_000_000):
    """Step until the relative change of u and T over `chunk` steps is below tol."""
    sim.residual()
    while sim.time < max_steps:
        sim.step(chunk)
        ru, rT = sim.residual()
        if max(ru, rT) < tol:
            return sim.time
    raise AssertionError(f"no steady state after {sim.time} steps (r_u={ru:.2e}, r_T={rT:.2e})")


def _table1():
    rows = []
    for line in open(os.path.join(GOLD, "table1_nusselt.txt")):
        if line.startswith("#") or not line.strip():
            continue
        da, ra, a, b, c = line.split()
        rows.append((float(da), float(ra), {0.4: float(a), 0.6: float(b), 0.9: float(c)}))
    return rows


@pytest.mark.parametrize("Ra", [1e3, 1e4, 1e5])
@pytest.mark.parametrize("phi", [0.4, 0.6, 0.9])
def test_table1_da1e2_on_128(Ra, phi):
    """Table 1, Da = 1e-2, on the paper's 128^2 grid: steady mean Nusselt
    number of the hot wall within 1.5 % of the "Present" column."""
    want = [r for r in _table1() if r[0] == 1e-2 and r[1] == Ra][0][2][phi]
    _, sim = build(128, 128, phi, Ra=Ra, Da=1e-2, Pr=1.0, with_oracle=False)
    steady(sim)
    nu = sim.nusselt(0)
    assert abs(nu / want - 1) < 0.015, (nu, want)


def test_sigma_does_not_change_steady_nusselt():
    """Sec. 3.2 / Fig. 7: Ra 1e5, Da 1e-2, phi 0.6 -- the steady Nusselt number
    is the same for sigma = 0.5, 1, 2 (paper: 3.4429 for all)."""
    nus = []
    for sigma in (0.5, 1.0, 2.0):
        _, sim = build(128, 128, 0.6, Ra=1e5, Da=1e-2, Pr=1.0, sigma=sigma, with_oracle=False)
        steady(sim, chunk=4000, tol=1e-10, max_steps=8_000_000)
        nus.append(sim.nusselt(0))
    assert max(nus) - min(nus) < 1e-6 * nus[1], nus
    assert abs(nus[1] / 3.4429 - 1) < 0.015


def test_brinkman_channel_1024x256_closed_form():
    """Body-force-driven porous channel, eps 0.5, Da 1e-2, periodic in x,
    walls on y = 0 and y = 255, Forchheimer term off: the steady profile is
    u(y) = (G K / nu)[1 - cosh(r (y - H/2)) / cosh(r H/2)],
    r^2 = phi nu / (nu_e K).  Relative L2 error (Eq. 45) below 1e-4
    (second order from 9.6e-4 at 65 nodes across)."""
    nx, ny = 1024, 256
    H, tau, phi, Da = ny - 1, 0.8, 0.5, 1e-2
    nu = (tau - 0.5) / 3
    G = 0.1 / H ** 2
    _, sim = build(nx, ny, phi, Ra=0.0, Da=Da, nu=nu, ax=G, forchheimer=False, kind=CHANNEL_X,
                   T=(None,) * 4, with_oracle=False)
    steady(sim, chunk=5000, tol=1e-11)
    _, ux, uy, _ = sim.macros()
    lat = sim.lattice
    y = np.arange(ny, dtype=float)
    r = math.sqrt(phi * lat.nu / (lat.nu_e * lat.K))
    ua = G * lat.K / lat.nu * (1 - np.cosh(r * (y - H / 2)) / np.cosh(r * H / 2))
    assert np.abs(uy).max() < 1e-12
    assert np.abs(ux - ux[:, :1]).max() < 1e-14
    err = math.sqrt(np.sum((ux[:, 0] - ua) ** 2)) / math.sqrt(np.sum(ua ** 2))
    assert err < 1e-4, err
