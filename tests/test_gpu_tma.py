"""The TMA-fed interior of the FP16N step against the per-thread kernel.

Both paths load the same stored values (the TMA one through bulk tensor
copies into shared memory, the other straight from global memory) and run
the same collision and store code, so every state they reach must be the
same bit for bit -- on walled and periodic sides, ragged widths (partial
tiles, pairs at the seams) and grids smaller than one tile.  The bounded
wait of the TMA path is checked on its failure branch: a wait on a barrier
that nothing completes must be reported as CLB_ERR_TIMEOUT and leave the
simulation intact.
"""
import numpy as np
import pytest

from cases import CAVITY, CHANNEL_X, PERIODIC, build
from paper_2110_05943_gb300 import clb
from paper_2110_05943_gb300.inputs import porosity_field

pytestmark = pytest.mark.gpu
F16N = 2
WALLS_X = ("wall", "wall", "periodic", "periodic")   # walls W/E, periodic S/N: rows 0 and ny - 1 wrap


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _pair(kind, nx, ny, seed):
    phi = porosity_field(nx, ny, seed=seed, ell=6.0, lo=0.4, span=0.5)
    hot = (1.0, 0.0, None, None) if kind[0] == "wall" else (None,) * 4
    ax = 0.0 if kind[0] == "wall" else 2e-6
    kw = dict(Ra=1e5, Da=1e-3, Pr=0.71, sigma=0.8, precision=F16N, kind=kind, T=hot, ax=ax, with_oracle=False)
    _, a = build(nx, ny, phi, **kw)
    _, b = build(nx, ny, phi, **kw)
    a.set_tma(True)
    b.set_tma(False)
    return a, b


@pytest.mark.parametrize("kind,nx,ny", [
    (CAVITY, 300, 37),      # ragged: a partial tile in x and in y
    (CAVITY, 128, 66),      # whole tiles (64 x 4 nodes over rows 1 .. 64)
    (CAVITY, 6, 5),         # smaller than one tile: a single interior pair per row
    (CHANNEL_X, 200, 21),   # periodic x: the seam pairs stay with the per-thread kernel
    (PERIODIC, 96, 40),     # periodic y: rows 0 and ny - 1 too (one-row blocks: one thread takes both)
    (PERIODIC, 512, 256),   # full 64 x 2-thread blocks: thread rows 0 and 1 take rows 0 and ny - 1
    (WALLS_X, 70, 33),
])
def test_tma_interior_matches_the_per_thread_path(kind, nx, ny):
    a, b = _pair(kind, nx, ny, seed=nx * 1000 + ny)
    for n in (1, 63, 200):   # single launches and captured graphs of 32 steps
        a.step(n)
        b.step(n)
        assert a.get_state() == b.get_state(), (kind, nx, ny, a.time)
    fa, fb = a.macros(), b.macros()
    assert all(np.array_equal(x, y) for x, y in zip(fa, fb))
    assert np.all(np.isfinite(fa[3])) and np.ptp(fa[1]) > 0.0   # a flow that moves


def test_tma_wait_expiry_is_reported_and_leaves_the_state_intact():
    a, b = _pair(CAVITY, 256, 130, seed=5)
    a.step(40)
    b.step(40)
    assert clb.clb_tma_selftest(a.handle, 20_000) == clb.CLB_ERR_TIMEOUT
    a.sync()                  # the flag was read and cleared by the self-test
    a.step(40)
    b.step(40)
    assert a.get_state() == b.get_state()


def test_tma_path_refused_where_it_does_not_exist():
    _, s = build(32, 32, 0.6, precision=0, with_oracle=False)       # FP64 form
    assert clb.load().clb_set_tma(s.handle, 1) == clb.CLB_ERR_ARG
    assert clb.load().clb_set_tma(s.handle, 0) == clb.CLB_OK
    assert clb.clb_tma_selftest(s.handle, 1000) == clb.CLB_ERR_ARG
