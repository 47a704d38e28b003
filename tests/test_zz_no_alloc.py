"""The allocation-free Nusselt reduction, clb_nusselt_field_static.

Some callers cannot call cudaMalloc: code running inside another
framework's memory pool that already holds the device memory, or loops that
cannot afford an allocation's device-wide synchronisation.  For them the
library offers a Nusselt reduction whose scratch is a fixed array in the
library's own device memory.  These tests call it through the C ABI and
check it against the ordinary, allocating clb_nusselt of the same state.

This file is named to be collected last, so that a run stopping at the
first failure has already run everything else; it also passes on its own in
a fresh process.
"""
import pytest

from cases import build

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_static_nusselt_matches_clb_nusselt_on_consecutive_calls(torch):
    from paper_2110_05943_gb300 import clb
    from paper_2110_05943_gb300.inputs import porosity_field
    nx, ny = 300, 70                      # the S/N walls span two reduction blocks
    phi = porosity_field(nx, ny, seed=21, ell=8.0)
    _, sim = build(nx, ny, phi, Ra=1e5, Da=1e-2, Pr=0.71, with_oracle=False)
    L = sim.lattice.L
    T = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for rnd, sides in enumerate(((clb.W, clb.S), (clb.E, clb.N))):
        sim.step(400)
        clb.clb_macros_device(sim.handle, None, None, None, T.data_ptr())
        # two calls in a row, sharing the one scratch array
        for k, side in enumerate(sides):
            clb.clb_nusselt_field_static(T.data_ptr(), nx, ny, side, L, 1.0, out.data_ptr() + 8 * (2 * rnd + k))
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for k, side in enumerate(sides):
            want = sim.nusselt(side)
            assert abs(got[2 * rnd + k] - want) <= TOL * max(1.0, abs(want)), (side, got[2 * rnd + k], want)
    sim.close()


def test_static_nusselt_on_a_caller_stream(torch):
    """The stream argument is honoured: two calls in a row on a
    non-default stream (ordered on it, so they share the scratch safely),
    and only that stream is synchronised before the results are read."""
    from paper_2110_05943_gb300 import clb
    from paper_2110_05943_gb300.inputs import porosity_field
    nx, ny = 130, 300                     # the W/E walls span two reduction blocks
    phi = porosity_field(nx, ny, seed=5, ell=6.0)
    _, sim = build(nx, ny, phi, Ra=1e5, Da=1e-2, Pr=0.71, with_oracle=False)
    sim.step(300)
    T = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    clb.clb_macros_device(sim.handle, None, None, None, T.data_ptr())
    torch.cuda.synchronize()              # T and out are ready before the other stream reads them
    s = torch.cuda.Stream()
    for k, side in enumerate((clb.W, clb.E)):
        clb.clb_nusselt_field_static(T.data_ptr(), nx, ny, side, sim.lattice.L, 1.0, out.data_ptr() + 8 * k,
                                     stream=s.cuda_stream)
    s.synchronize()
    got = out.cpu().numpy()
    for k, side in enumerate((clb.W, clb.E)):
        want = sim.nusselt(side)
        assert abs(got[k] - want) <= TOL * max(1.0, abs(want)), (side, got[k], want)
    sim.close()


def test_static_nusselt_rejects_walls_beyond_its_scratch(torch):
    """A wall longer than CLB_STATIC_MAX_WALL nodes is refused on the host
    before any kernel is launched."""
    from paper_2110_05943_gb300 import clb
    T = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(clb.ClbError) as e:
        clb.clb_nusselt_field_static(T.data_ptr(), 1024 * 256 + 1, 3, clb.S, 10.0, 1.0, out.data_ptr())
    assert e.value.code == clb.CLB_ERR_ARG
    with pytest.raises(clb.ClbError):
        clb.clb_nusselt_field_static(T.data_ptr(), 8, 1, clb.S, 10.0, 1.0, out.data_ptr())
