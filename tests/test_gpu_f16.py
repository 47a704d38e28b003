"""The reduced-precision forms against the FP64 oracle and the FP64 GPU path.

CLB_F16S stores each distribution in FP16 as its deviation from the rest
state; CLB_F16N as its deviation from the local equilibrium of the node
that wrote it (that node's rho, u, T stored in FP16 as the baseline).  Both
compute in FP32.  Bounds are measured errors times ~4 (recorded beside each
check); the target for a converged run is the FP64 mean Nusselt number
within 1e-4 relative.
"""
import numpy as np
import pytest

from cases import CAVITY, PERIODIC, build, field_errors

pytestmark = pytest.mark.gpu
F16S, F16N = 1, 2


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def steady(sim, chunk=2000, tol=1e-8, max_steps=3_000_000):
    sim.residual()
    while sim.time < max_steps:
        sim.step(chunk)
        ru, rT = sim.residual()
        if max(ru, rT) < tol:
            break
    return sim.time


def test_f16n_cavity_64_10k_steps_vs_oracle():
    """64^2 cavity, 10,000 steps: fields and Nusselt number of the FP16N form
    against the FP64 oracle, within FP16 storage resolution."""
    orc, sim = build(64, 64, 0.6, Ra=1e4, Da=1e-2, Pr=1.0, precision=F16N)
    orc.step(10_000)
    sim.step(10_000)
    e = field_errors(sim.macros(), orc.macros())
    assert e["rho-1"] < 6e-3 and e["ux"] < 2e-3 and e["uy"] < 2e-3 and e["T"] < 1e-4, e
    assert abs(sim.nusselt(0) / orc.nusselt(0) - 1) < 2e-5


def test_f16n_random_porosity_ragged_vs_oracle():
    """300 x 37 seeded-porosity cavity, 1,500 steps, against the oracle."""
    from paper_2110_05943_gb300.inputs import porosity_field
    phi = porosity_field(300, 37, seed=11, ell=8.0)
    orc, sim = build(300, 37, phi, Ra=1e6, Da=1e-3, Pr=0.71, sigma=0.8, precision=F16N)
    orc.step(1500)
    sim.step(1500)
    e = field_errors(sim.macros(), orc.macros())
    assert e["rho-1"] < 2e-2 and e["ux"] < 4e-3 and e["uy"] < 4e-3 and e["T"] < 7e-4, e


@pytest.mark.parametrize("prec,u_uc,dT,nu", [
    (F16N, 1e-3, 5e-4, 1e-3),   # bench at 2048^2 / 30,000 steps: 3.5e-5, 3.3e-5, 2.3e-5
    (F16S, 2e-3, 5e-3, 3e-2),   # bench at 2048^2 / 30,000 steps: 8.7e-5, 6.2e-4, 2.6e-3
])
def test_f16_forms_on_full_size_blocks_vs_fp64(prec, u_uc, dT, nu):
    """512^2 seeded cavity (Ra 1e6, Da 1e-3, Pr 0.71, sigma 0.8), 4,000
    steps, against the FP64 GPU path (parity-tested against the oracle): the
    grid is large enough for the pair step's full 64 x 2-thread blocks (the
    smaller grids above run one-row blocks).  Max |u - u64| over the velocity
    scale u_c = Ma c_s of Eq. 46, max |T - T64| (dT = 1), relative Nu."""
    from paper_2110_05943_gb300.inputs import porosity_field
    n = 512
    phi = porosity_field(n, n, seed=512, ell=16.0)
    kw = dict(Ra=1e6, Da=1e-3, Pr=0.71, sigma=0.8, with_oracle=False)
    _, s64 = build(n, n, phi, **kw)
    _, s16 = build(n, n, phi, precision=prec, **kw)
    s64.step(4000)
    s16.step(4000)
    a, b = s16.macros(), s64.macros()
    uc = 0.1 / np.sqrt(3.0)
    eu = max(float(np.max(np.abs(a[k] - b[k]))) for k in (1, 2)) / uc
    eT = float(np.max(np.abs(a[3] - b[3])))
    en = abs(s16.nusselt(0) / s64.nusselt(0) - 1)
    assert np.all(np.isfinite(a[3])) and float(np.max(np.abs(b[1]))) > 1e-6, "no flow to compare"
    assert eu < u_uc and eT < dT and en < nu, (prec, eu, eT, en)


def test_f16n_steady_nusselt_within_1e4_of_fp64():
    """Table 1 row Da 1e-2, Ra 1e4, phi 0.6 on 128^2: steady mean Nusselt
    number of the FP16N form within 1e-4 of the FP64 path."""
    _, s64 = build(128, 128, 0.6, Ra=1e4, Da=1e-2, Pr=1.0, with_oracle=False)
    _, s16 = build(128, 128, 0.6, Ra=1e4, Da=1e-2, Pr=1.0, precision=F16N, with_oracle=False)
    steady(s64, tol=1e-10)
    steady(s16, tol=1e-6, max_steps=1_000_000)
    assert abs(s16.nusselt(0) / s64.nusselt(0) - 1) < 1e-4


def _mean_nu(sim, steps, window=20, every=2500):
    sim.step(steps - window * every)
    vals = []
    for _ in range(window):
        sim.step(every)
        vals.append(sim.nusselt(0))
    return float(np.mean(vals))


@pytest.mark.slow
def test_fp16_forms_unbiased_at_high_rayleigh():
    """128^2 cavity, Ra 1e6, Da 1e-3, phi 0.6, sigma 0.8, 400,000 steps: the
    mean hot-wall Nusselt number over the last 50,000 steps.  With unbiased
    (stochastic) rounding of the stored values the FP16N form stays within
    1e-4 of FP64 (round-to-nearest left 1e-3: the state-correlated rounding
    acts as a steady heat source), and the rest-shifted form within 1 %
    (round-to-nearest: 72-130 % off at Ra 1e4-1e5 on 128^2)."""
    runs = {}
    for prec in (0, F16N, F16S):
        _, s = build(128, 128, 0.6, Ra=1e6, Da=1e-3, Pr=0.71, sigma=0.8, precision=prec, with_oracle=False)
        runs[prec] = _mean_nu(s, 400_000)
    assert abs(runs[F16N] / runs[0] - 1) < 1e-4, runs
    assert abs(runs[F16S] / runs[0] - 1) < 1e-2, runs


@pytest.mark.slow
def test_f16n_conduction_dominated_case_unbiased():
    """128^2, Ra 1e5, Da 1e-4, phi 0.4, 400,000 steps: a slow, conduction-
    dominated cavity in which FP32 rounding of O(0.1) thermal distributions
    used to bias Nu by 8.6e-4; with the rest-centred thermal arithmetic the
    FP16N form stays within 1e-4 of FP64 (measured 2.3e-6 at 600,000 steps)."""
    runs = {}
    for prec in (0, F16N):
        _, s = build(128, 128, 0.4, Ra=1e5, Da=1e-4, Pr=0.71, precision=prec, with_oracle=False)
        runs[prec] = _mean_nu(s, 400_000)
    assert abs(runs[F16N] / runs[0] - 1) < 1e-4, runs


@pytest.mark.parametrize("shift,forch", [(False, True), (True, False)])
def test_f16n_variants_track_oracle(shift, forch):
    from paper_2110_05943_gb300.inputs import porosity_field
    phi = porosity_field(40, 40, seed=2, ell=6.0)
    orc, sim = build(40, 40, phi, Ra=1e5, Da=1e-2, Pr=0.71, shift=shift, forchheimer=forch, precision=F16N)
    orc.step(2000)
    sim.step(2000)
    e = field_errors(sim.macros(), orc.macros())
    assert e["ux"] < 5e-3 and e["uy"] < 5e-3 and e["T"] < 5e-4, e


def test_f16s_tracks_oracle_over_short_times():
    """The rest-shifted form is within FP16 resolution of the oracle for a
    short transient (200 steps on a 64^2 cavity)."""
    orc, sim = build(64, 64, 0.6, Ra=1e4, Da=1e-2, Pr=1.0, precision=F16S)
    orc.step(200)
    sim.step(200)
    e = field_errors(sim.macros(), orc.macros())
    assert e["T"] < 5e-3 and e["ux"] < 5e-2, e


@pytest.mark.parametrize("prec", [F16S, F16N])
def test_f16_periodic_set_fields_and_checkpoint(prec):
    """Periodic domain from smooth random fields: the initial macros
    reproduce the given fields to FP16 resolution, and a checkpoint
    resumes bit for bit."""
    from paper_2110_05943_gb300.inputs import smooth_fields
    nx, ny = 50, 40
    rho, ux, uy, T = smooth_fields(nx, ny, seed=9)
    _, sim = build(nx, ny, 0.7, Ra=1e5, Da=1e-2, Pr=0.71, sigma=1.3, L=32, kind=PERIODIC, T=(None,) * 4,
                   precision=prec, with_oracle=False)
    sim.set_fields(rho, ux, uy, T)
    r0, u0, v0, T0 = sim.macros()
    assert np.abs(T0 - T).max() < 2e-3 and np.abs(u0 - ux).max() < 2e-4
    sim.step(123)
    st = sim.get_state()
    sim.step(50)
    a = sim.macros()
    sim.set_state(st)
    sim.step(50)
    b = sim.macros()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_f16n_small_grids_and_corners():
    for nx, ny in ((4, 4), (5, 33), (33, 5)):
        orc, sim = build(nx, ny, 0.7, Ra=1e4, Da=1e-2, precision=F16N)
        orc.step(300)
        sim.step(300)
        e = field_errors(sim.macros(), orc.macros())
        assert e["T"] < 1e-3 and np.isfinite(list(e.values())).all(), (nx, ny, e)
