"""Batched form: independent cases advanced together, one launch per step
(graph mode) or one persistent launch per 32 steps (persistent mode).

Each case runs the same per-node code as a single simulation, so after the
same number of steps a batched case must equal its stand-alone run bit for
bit -- in every storage form, whatever tile shape the tuner picks, and with
other cases retired part-way.  One case is also checked against the oracle.
"""
import numpy as np
import pytest

from cases import build, field_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cases(prec):
    from paper_2110_05943_gb300 import clb
    from paper_2110_05943_gb300.inputs import porosity_field
    spec = [  # nx, ny, Ra, Da, Pr, sigma, phi (None: random field)
        (37, 21, 1e5, 1e-2, 0.71, 0.8, 0.6),
        (64, 64, 1e4, 1e-2, 1.0, 1.0, 0.6),
        (130, 40, 1e6, 1e-3, 0.71, 1.5, None),
        (20, 90, 1e3, 1e-4, 0.71, 0.5, 0.45),
        (9, 9, 1e5, 1e-1, 0.71, 2.0, 0.9),
    ]
    params, phis = [], []
    for k, (nx, ny, Ra, Da, Pr, sg, phi) in enumerate(spec):
        params.append(clb.clb_params_default(nx=nx, ny=ny, Ra=Ra, Da=Da, Pr=Pr, sigma=sg, precision=prec))
        phis.append(porosity_field(nx, ny, seed=30 + k, ell=6.0) if phi is None else phi)
    return spec, params, phis


def _single(params, phi):
    from paper_2110_05943_gb300 import clb
    return clb.Simulation.create(params, phi, clb.clb_bc_cavity(1.0, 0.0))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batch_equals_single_runs_bit_for_bit(prec):
    from paper_2110_05943_gb300 import clb
    spec, params, phis = _cases(prec)
    batch = clb.Batch(params, phis, [clb.clb_bc_cavity(1.0, 0.0) for _ in params])
    batch.step(77)
    for c, (p, phi) in enumerate(zip(params, phis)):
        s = _single(p, phi)
        s.step(77)
        for a, b in zip(batch.macros(c), s.macros()):
            assert np.array_equal(a, b), (prec, c)
        s.close()
    nu = batch.nusselt(0)
    assert np.isfinite(nu).all() and nu.shape == (len(params),)
    assert batch.nodes == sum(p.nx * p.ny for p in params)
    batch.close()


def test_batch_case_matches_oracle():
    from paper_2110_05943_gb300 import clb
    spec, params, phis = _cases(0)
    batch = clb.Batch(params, phis, [clb.clb_bc_cavity(1.0, 0.0) for _ in params])
    batch.step(600)
    import oracle
    c = 2
    nx, ny, Ra, Da, Pr, sg, _ = spec[c]
    o = oracle.Oracle(oracle.Problem(nx=nx, ny=ny, Ra=Ra, Da=Da, Pr=Pr, sigma=sg), phi=phis[c])
    o.step(600)
    e = field_errors(batch.macros(c), o.macros())
    assert all(v <= 1e-10 for v in e.values()), e
    batch.close()


@pytest.mark.parametrize("prec", [0, 2])
def test_retired_cases_freeze_and_tuning_keeps_results(prec):
    from paper_2110_05943_gb300 import clb
    spec, params, phis = _cases(prec)
    n = len(params)
    batch = clb.Batch(params, phis, [clb.clb_bc_cavity(1.0, 0.0) for _ in params])
    batch.step(40)
    frozen = batch.macros(1)
    active = [1] * n
    active[1] = 0
    batch.set_active(active)
    choice = batch.tune(steps=2)          # 12 tilings x 3 steps = 36 more steps for the active cases
    assert 0 <= choice < 12
    batch.step(33)
    for a, b in zip(batch.macros(1), frozen):
        assert np.array_equal(a, b)
    total = 40 + 36 + 33
    for c in (0, 2, 4):
        s = _single(params[c], phis[c])
        s.step(total)
        for a, b in zip(batch.macros(c), s.macros()):
            assert np.array_equal(a, b), (prec, c)
        s.close()
    # 69 batch steps (an odd count) after retirement: the case resumes from its own buffer
    batch.set_active([1] * n)
    batch.step(11)
    s = _single(params[1], phis[1])
    s.step(40 + 11)
    for a, b in zip(batch.macros(1), s.macros()):
        assert np.array_equal(a, b), prec
    s.close()
    batch.close()


@pytest.mark.parametrize("prec", [0, 2])
def test_every_tiling_gives_the_same_bits(prec):
    """Five steps under each of the 12 tilings in turn (four block shapes,
    4/16/64 tiles per CTA) equal 60 stand-alone steps."""
    from paper_2110_05943_gb300 import clb
    spec, params, phis = _cases(prec)
    batch = clb.Batch(params, phis, [clb.clb_bc_cavity(1.0, 0.0) for _ in params])
    for choice in range(12):
        batch.set_tiling(choice)
        batch.step(5)
    with pytest.raises(clb.ClbError):
        batch.set_tiling(12)
    for c, (p, phi) in enumerate(zip(params, phis)):
        s = _single(p, phi)
        s.step(60)
        for a, b in zip(batch.macros(c), s.macros()):
            assert np.array_equal(a, b), (prec, c)
        s.close()
    batch.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_persistent_mode_equals_graph_mode_bit_for_bit(prec):
    """The persistent launch (grid barrier between steps, coherent L2 loads)
    runs the same per-node code: after 77 steps (two 32-step graphs and a
    13-step launch) every case equals the graph-mode batch bit for bit, and
    switching modes mid-run changes nothing either."""
    from paper_2110_05943_gb300 import clb
    spec, params, phis = _cases(prec)
    bcs = [clb.clb_bc_cavity(1.0, 0.0) for _ in params]
    ref = clb.Batch(params, phis, bcs)
    per = clb.Batch(params, phis, bcs)
    mix = clb.Batch(params, phis, bcs)
    ref.set_mode(clb.CLB_BATCH_GRAPH)
    per.set_mode(clb.CLB_BATCH_PERSISTENT)
    mix.set_mode(clb.CLB_BATCH_GRAPH)
    ref.step(77)
    per.step(77)
    mix.step(33)
    mix.set_mode(clb.CLB_BATCH_PERSISTENT)
    mix.step(44)
    for c in range(len(params)):
        want = ref.macros(c)
        for other in (per, mix):
            for a, b in zip(other.macros(c), want):
                assert np.array_equal(a, b), (prec, c)
    assert per.time == 77 and mix.time == 77
    for b in (ref, per, mix):
        b.close()


def test_persistent_barrier_wait_expires_and_reports_timeout():
    """Failure detection of the persistent mode: a step whose grid barrier
    waits for one block more than the launch has (a flag nothing sets)
    gives up after ~1 ms of SM clock, every block returns, and the call
    reports CLB_ERR_TIMEOUT.  The context and the batch stay usable: the
    state was not advanced, and stepping on gives the same bits as a batch
    that never ran the test."""
    from paper_2110_05943_gb300 import clb
    spec, params, phis = _cases(2)
    bcs = [clb.clb_bc_cavity(1.0, 0.0) for _ in params]
    a = clb.Batch(params, phis, bcs)
    ref = clb.Batch(params, phis, bcs)
    a.set_mode(clb.CLB_BATCH_PERSISTENT)
    a.step(40)
    ref.step(40)
    assert a.barrier_selftest(2_000_000) == clb.CLB_ERR_TIMEOUT
    assert a.time == 40
    a.sync()                                  # the flag was reported once and cleared
    a.step(24)
    ref.step(24)
    for c in range(len(params)):
        for x, y in zip(a.macros(c), ref.macros(c)):
            assert np.array_equal(x, y), c
    assert a.barrier_selftest(0) == clb.CLB_ERR_ARG          # bound outside 1 .. 4e9
    a.close()
    ref.close()
