"""The C ABI library builds for sm_103a, loads without a GPU, and exports
every entry point include/*.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header=None):
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h") or (header and h != header):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(clb_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared("clb.h")
    for n in ("clb_init", "clb_step", "clb_macros", "clb_nusselt", "clb_residual", "clb_destroy",
              "clb_get_state", "clb_set_state", "clb_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2110_05943_gb300 import clb
    lib = clb.load()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_params_default_and_abi_struct_sizes():
    from paper_2110_05943_gb300 import clb
    p = clb.clb_params_default()
    assert (p.nx, p.ny) == (64, 64) and p.Ra == 1e4 and p.s3 == 1.2 and p.s4 == 1.8 and p.Ma == 0.1
    assert ctypes.sizeof(clb.ClbParams) == 6 * 4 + 18 * 8
    bc = clb.clb_bc_cavity(1.0, 0.0)
    assert list(bc.kind) == [1, 1, 1, 1] and list(bc.thermal) == [1, 1, 0, 0]


def test_init_rejects_bad_arguments_before_touching_the_gpu():
    """Argument validation happens on the host first; these calls fail with
    CLB_ERR_ARG whether or not a GPU is present."""
    import numpy as np
    import pytest
    from paper_2110_05943_gb300 import clb
    bc = clb.clb_bc_cavity()
    p = clb.clb_params_default(nx=16, ny=16)
    with pytest.raises(clb.ClbError) as e:
        clb.clb_init(p, np.full(256, 1.5), bc)        # porosity > 1
    assert e.value.code == clb.CLB_ERR_ARG
    with pytest.raises(clb.ClbError):
        clb.clb_init(clb.clb_params_default(nx=3, ny=16), np.full(48, 0.5), bc)   # walled dim < 4
    with pytest.raises(clb.ClbError):
        clb.clb_init(clb.clb_params_default(nx=16, ny=16, Da=-1.0), np.full(256, 0.5), bc)
    with pytest.raises(clb.ClbError):
        clb.clb_init(clb.clb_params_default(nx=16, ny=16, Ra=0.0), np.full(256, 0.5), bc)  # Eq. 46 needs Ra
    mixed = clb.clb_bc(("wall", "periodic", "wall", "wall"))
    with pytest.raises(clb.ClbError):
        clb.clb_init(p, np.full(256, 0.5), mixed)


def test_fp16_grid_size_limit_checked_before_phi_is_read():
    """The FP16 forms index with 32-bit offsets: 9 * ny * pitch must stay
    below 2^31.  The limit is checked on the host before the porosity array
    is read, so a one-value array stands in for the 16384 x 14564 field."""
    import ctypes as C
    import numpy as np
    from paper_2110_05943_gb300 import clb
    lib = clb.load()
    bc = clb.clb_bc_cavity()
    one = np.full(1, 0.5)
    h = C.c_void_p()
    for prec, nx, ny in ((clb.CLB_F16N, 16384, 14564), (clb.CLB_F16S, 16385, 14600)):
        p = clb.clb_params_default(nx=nx, ny=ny, precision=prec)
        rc = lib.clb_init(C.byref(h), C.byref(p), one.ctypes.data_as(C.POINTER(C.c_double)), None, C.byref(bc), None)
        assert rc == clb.CLB_ERR_ARG and not h.value
        assert b"32-bit" in lib.clb_last_error(None)


def test_surrogate_entry_points_declared_and_reject_bad_shapes():
    """The learned warm start's kernels (include/clb_nop.h) are exported and
    validate shapes on the host before any launch."""
    from paper_2110_05943_gb300 import surrogate
    names = _declared("clb_nop.h")
    for n in ("clb_nop_conv_fwd", "clb_nop_conv_dgrad", "clb_nop_conv_wgrad", "clb_nop_adam", "clb_nop_mse"):
        assert n in names
    lib = surrogate._lib()
    fake = ctypes.c_void_p(16)          # never dereferenced: the calls fail validation first
    assert lib.clb_nop_conv_fwd(fake, fake, None, None, fake, 0, 1, 1, 8, 8, 4, 4, 5, None) == -1      # taps 5
    assert lib.clb_nop_conv_fwd(fake, fake, None, None, fake, 0, 1, 0, 8, 8, 4, 4, 9, None) == -1      # n = 0
    assert lib.clb_nop_conv_fwd(None, fake, None, None, fake, 0, 1, 1, 8, 8, 4, 4, 9, None) == -1      # null x
    # 32-bit index guard: 2^16 x 2^16 pixels x 1 channel x 9 taps
    assert lib.clb_nop_conv_fwd(fake, fake, None, None, fake, 0, 1, 1, 65536, 65536, 1, 1, 9, None) == -1
    assert lib.clb_nop_pool2(fake, fake, 1, 7, 8, 4, 0, None) == -1                            # odd height
    assert lib.clb_nop_adam(fake, fake, fake, fake, None, 10, 1e-3, 0.9, 0.999, 1e-8, 0, None) == -1  # t = 0


def test_non_finite_inputs_rejected_on_the_host():
    """NaN or infinite porosity, parameters or row forces are argument
    errors (CLB_ERR_ARG) found before any CUDA call, so they never reach a
    kernel."""
    import numpy as np
    import pytest
    from paper_2110_05943_gb300 import clb
    bc = clb.clb_bc_cavity()
    p = clb.clb_params_default(nx=16, ny=16)
    for bad in (np.nan, np.inf, -np.inf, 0.0, -0.5):
        phi = np.full(256, 0.5)
        phi[37] = bad
        with pytest.raises(clb.ClbError) as e:
            clb.clb_init(p, phi, bc)
        assert e.value.code == clb.CLB_ERR_ARG
    for field in ("Ra", "Da", "Pr", "sigma", "dT", "s3", "varpi"):
        q = clb.clb_params_default(nx=16, ny=16)
        setattr(q, field, float("nan"))
        with pytest.raises(clb.ClbError) as e:
            clb.clb_init(q, np.full(256, 0.5), bc)
        assert e.value.code == clb.CLB_ERR_ARG, field
    ay = np.zeros(16)
    ay[3] = np.nan
    with pytest.raises(clb.ClbError) as e:
        clb.clb_init(p, np.full(256, 0.5), bc, ay_row=ay)
    assert e.value.code == clb.CLB_ERR_ARG
