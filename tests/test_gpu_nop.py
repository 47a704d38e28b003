"""Learned warm start: the library's BF16 tensor-core kernels against plain
PyTorch FP32 CPU references of the same operations, on BF16-representable
inputs (so every product is exact and only the FP32 summation order and the
final BF16 rounding differ), and the whole network's forward and backward
pass against PyTorch autograd."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
F = torch.nn.functional


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2110_05943_gb300 import surrogate
    return surrogate._lib()


def _bf(shape, seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(shape, generator=g) * scale).to(torch.bfloat16)


def _p(t):
    return None if t is None else t.data_ptr()


def _ref_conv(x_nhwc, wmat, taps, cin, cout, bias=None):
    """FP32 CPU reference: x (n,h,w,cin), wmat [taps*cin][cout] -> (n,h,w,cout)."""
    k = 3 if taps == 9 else 1
    w = wmat.float().reshape(k, k, cin, cout).permute(3, 2, 0, 1)       # (cout, cin, ky, kx)
    y = F.conv2d(x_nhwc.float().permute(0, 3, 1, 2), w, bias, padding=k // 2)
    return y.permute(0, 2, 3, 1)


def _close(a, b, rel):
    a, b = a.float(), b.float()
    err = (a - b).abs().max().item()
    scale = b.abs().max().item() + 1e-30
    assert err <= rel * scale, (err, scale, err / scale)


SHAPES = [  # n, h, w, cin, cout, taps: ragged against the 64 x 64 x 32 (mma.sync) and 128 x N x 64 (tcgen05) tiles
    (2, 12, 20, 7, 24, 9),         # cin 7: forward on mma.sync; input gradient (cout 24) on tcgen05
    (1, 16, 16, 40, 72, 9),
    (3, 8, 10, 24, 3, 1),          # 1x1, N = 3 padded to 16 on tcgen05; cout 3: input gradient on mma.sync
    (2, 6, 6, 130, 20, 9),         # neither channel count a multiple of 8: mma.sync both ways
    (2, 12, 20, 8, 24, 9),
    (1, 8, 8, 288, 96, 9),         # input gradient N = 288: two N tiles (256 + 32)
    (2, 10, 6, 24, 192, 9),
    (3, 16, 12, 48, 96, 9),
    # whole-row tiles of 128 pixels: the TMA-fed path (channels zero-filled
    # up to 64-wide chunks, image borders zero-filled by the loads)
    (2, 8, 128, 24, 24, 9),        # W = 128, C = 24 < 64
    (2, 8, 128, 8, 24, 9),         # the input layer's 8 channels
    (1, 16, 64, 48, 96, 9),        # W = 64: tiles of 2 rows
    (2, 16, 32, 96, 48, 9),        # W = 32, C = 96: two channel chunks
    (2, 8, 128, 72, 24, 9),        # C = 72: 64 + 8
    (1, 16, 16, 288, 96, 9),       # W = 16, C = 288; input gradient N = 288: two N tiles
    (1, 8, 128, 24, 8, 1),         # 1x1 convolution
]
# A production layer: the training batch (16 x 128^2), 24 -> 24 channels.
PRODUCTION = (16, 128, 128, 24, 24, 9)


@pytest.mark.parametrize("shape", SHAPES + [PRODUCTION])
@pytest.mark.parametrize("relu", [0, 1])
def test_conv_forward(lib, shape, relu):
    n, h, w, cin, cout, taps = shape
    x, wm = _bf((n, h, w, cin), 1), _bf((taps * cin, cout), 2, 1.0 / math.sqrt(taps * cin))
    b = torch.randn(cout, generator=torch.Generator().manual_seed(3))
    ref = _ref_conv(x, wm, taps, cin, cout, b)
    if relu:
        ref = ref.clamp_min(0)
    xd, wd, bd = x.cuda(), wm.cuda(), b.cuda()
    wt = wm.t().contiguous().cuda()
    for wtp in (None, wt):             # mma.sync path, then tcgen05 where the shape allows
        y32 = torch.empty((n, h, w, cout), device="cuda")
        assert lib.clb_nop_conv_fwd(_p(xd), _p(wd), _p(wtp), _p(bd), _p(y32), 1, relu, n, h, w, cin, cout, taps,
                                    None) == 0
        assert lib.clb_nop_check(None) == 0
        _close(y32.cpu(), ref, 1e-5)
        y16 = torch.empty((n, h, w, cout), device="cuda", dtype=torch.bfloat16)
        assert lib.clb_nop_conv_fwd(_p(xd), _p(wd), _p(wtp), _p(bd), _p(y16), 0, relu, n, h, w, cin, cout, taps,
                                    None) == 0
        _close(y16.cpu(), ref, 8e-3)


# the network's head (1x1, 24 -> 4): weight and input gradients on CUDA-core
# kernels, small and at the training batch
HEADS = [(2, 8, 12, 24, 4, 1), (3, 5, 7, 8, 4, 1), (16, 128, 128, 24, 4, 1)]


@pytest.mark.parametrize("shape", SHAPES + [PRODUCTION] + HEADS)
def test_conv_input_gradient(lib, shape):
    n, h, w, cin, cout, taps = shape
    x = _bf((n, h, w, cin), 4)
    wm, dy = _bf((taps * cin, cout), 5), _bf((n, h, w, cout), 6)
    xr = x.float().requires_grad_(True)
    _ref_conv(xr, wm, taps, cin, cout).backward(dy.float())
    ref = xr.grad * (x.float() > 0)
    dx = torch.empty((n, h, w, cin), device="cuda", dtype=torch.bfloat16)
    xd = x.cuda()
    assert lib.clb_nop_conv_dgrad(_p(dy.cuda()), _p(wm.cuda()), _p(xd), _p(dx), n, h, w, cin, cout, taps, None) == 0
    assert lib.clb_nop_check(None) == 0
    _close(dx.cpu(), ref, 8e-3)



@pytest.mark.parametrize("shape,splitk", [(s, k) for s in SHAPES for k in (1, 7)] + [(PRODUCTION, 0)] +
                         [(s, 0) for s in HEADS])
def test_conv_weight_gradient(lib, shape, splitk):
    """splitk 0 = the library's own split, as training calls it: on the
    production layer a single FP32 tensor-core accumulator over all 262,144
    pixels (splitk 1) drifts by ~3e-4, which is why the library splits."""
    n, h, w, cin, cout, taps = shape
    x, wm, dy = _bf((n, h, w, cin), 7), _bf((taps * cin, cout), 8), _bf((n, h, w, cout), 9)
    wr = wm.float().requires_grad_(True)
    _ref_conv(x, wr, taps, cin, cout).backward(dy.float())
    dw = torch.zeros((taps * cin, cout), device="cuda")
    assert lib.clb_nop_conv_wgrad(_p(x.cuda()), _p(dy.cuda()), _p(dw), n, h, w, cin, cout, taps, splitk, None) == 0
    _close(dw.cpu(), wr.grad, 1e-5)
    # the same pass with the bias gradient (a row of ones on the tensor-core path)
    dw2, db = torch.zeros_like(dw), torch.zeros(cout, device="cuda")
    assert lib.clb_nop_conv_wgrad_bias(_p(x.cuda()), _p(dy.cuda()), _p(dw2), _p(db), n, h, w, cin, cout, taps, splitk,
                                       None) == 0
    _close(dw2.cpu(), wr.grad, 1e-5)
    _close(db.cpu(), dy.double().sum(dim=(0, 1, 2)).float(), 1e-5)


def test_transpose(lib):
    w = _bf((37, 19), 30)
    wt = torch.empty((19, 37), device="cuda", dtype=torch.bfloat16)
    assert lib.clb_nop_transpose(_p(w.cuda()), _p(wt), 37, 19, None) == 0
    assert torch.equal(wt.cpu(), w.t())


@pytest.mark.parametrize("c,ca,cb,nadd", [(12, 5, 9, 1001), (24, 48, 24, 1000), (288, 96, 192, 4096)])
def test_bias_grad_pool_up_concat(lib, c, ca, cb, nadd):
    """c, ca, cb, nadd multiples of 8: the 16-byte (8-channel) kernels; otherwise the scalar ones."""
    n, h, w = 2, 10, 14
    dy = _bf((n, h, w, c), 10)
    db = torch.zeros(c, device="cuda")
    assert lib.clb_nop_bias_grad(_p(dy.cuda()), _p(db), n * h * w, c, None) == 0
    _close(db.cpu(), dy.float().sum(dim=(0, 1, 2)), 1e-6)

    x = _bf((n, h, w, c), 11)
    y = torch.empty((n, h // 2, w // 2, c), device="cuda", dtype=torch.bfloat16)
    assert lib.clb_nop_pool2(_p(x.cuda()), _p(y), n, h, w, c, 0, None) == 0
    ref = F.avg_pool2d(x.float().permute(0, 3, 1, 2), 2).permute(0, 2, 3, 1)
    _close(y.cpu(), ref, 8e-3)
    xr = x.float().requires_grad_(True)
    g = _bf((n, h // 2, w // 2, c), 12)
    F.avg_pool2d(xr.permute(0, 3, 1, 2), 2).permute(0, 2, 3, 1).backward(g.float())
    dx = torch.empty((n, h, w, c), device="cuda", dtype=torch.bfloat16)
    assert lib.clb_nop_pool2(_p(g.cuda()), _p(dx), n, h, w, c, 1, None) == 0
    _close(dx.cpu(), xr.grad, 1e-6)

    s = _bf((n, h, w, c), 13)
    u = torch.empty((n, 2 * h, 2 * w, c), device="cuda", dtype=torch.bfloat16)
    assert lib.clb_nop_up2(_p(s.cuda()), _p(u), n, h, w, c, 0, None) == 0
    sr = s.float().requires_grad_(True)
    ur = F.interpolate(sr.permute(0, 3, 1, 2), scale_factor=2, mode="nearest").permute(0, 2, 3, 1)
    _close(u.cpu(), ur.detach(), 0.0)
    gu = _bf((n, 2 * h, 2 * w, c), 14)
    ur.backward(gu.float())
    ds = torch.empty((n, h, w, c), device="cuda", dtype=torch.bfloat16)
    assert lib.clb_nop_up2(_p(gu.cuda()), _p(ds), n, h, w, c, 1, None) == 0
    _close(ds.cpu(), sr.grad, 8e-3)

    a, b = _bf((n * h * w, ca), 15), _bf((n * h * w, cb), 16)
    yy = torch.empty((n * h * w, ca + cb), device="cuda", dtype=torch.bfloat16)
    ad, bd = a.cuda(), b.cuda()
    assert lib.clb_nop_concat(_p(ad), _p(bd), _p(yy), n * h * w, ca, cb, 0, None) == 0
    assert torch.equal(yy.cpu(), torch.cat([a, b], dim=1))
    a2, b2 = torch.empty_like(ad), torch.empty_like(bd)
    assert lib.clb_nop_concat(_p(a2), _p(b2), _p(yy), n * h * w, ca, cb, 1, None) == 0
    assert torch.equal(a2.cpu(), a) and torch.equal(b2.cpu(), b)

    d1, d2, m = _bf((nadd,), 17), _bf((nadd,), 18), _bf((nadd,), 19)
    out = torch.empty((nadd,), device="cuda", dtype=torch.bfloat16)
    assert lib.clb_nop_add_mask(_p(d1.cuda()), _p(d2.cuda()), _p(m.cuda()), _p(out), nadd, None) == 0
    _close(out.cpu(), (d1.float() + d2.float()) * (m.float() > 0), 8e-3)
    assert lib.clb_nop_add_mask(_p(d1.cuda()), None, _p(m.cuda()), _p(out), nadd, None) == 0
    _close(out.cpu(), d1.float() * (m.float() > 0), 8e-3)


def test_bias_grad_production(lib):
    """The training batch's 128^2 x 16 images, 24 channels (grid-stride vector sums)."""
    npix, c = 16 * 128 * 128, 24
    dy = _bf((npix, c), 21)
    db = torch.zeros(c, device="cuda")
    assert lib.clb_nop_bias_grad(_p(dy.cuda()), _p(db), npix, c, None) == 0
    _close(db.cpu(), dy.double().sum(dim=0).float(), 1e-5)


def test_mse_and_adam(lib):
    n = 5000
    g = torch.Generator().manual_seed(20)
    pred, tgt = torch.randn(n, generator=g), torch.randn(n, generator=g)
    loss = torch.zeros(1, device="cuda")
    grad = torch.empty(n, device="cuda", dtype=torch.bfloat16)
    assert lib.clb_nop_mse(_p(pred.cuda()), _p(tgt.cuda()), None, 1, _p(grad), _p(loss), n, None) == 0
    assert abs(loss.item() - F.mse_loss(pred, tgt).item()) <= 1e-5 * F.mse_loss(pred, tgt).item()
    _close(grad.cpu(), 2 * (pred - tgt) / n, 8e-3)
    # channel weights: 5 channels fastest
    wch = torch.tensor([1.0, 0.5, 2.0, 0.0, 3.0])
    wfull = wch.repeat(n // 5)
    loss.zero_()
    assert lib.clb_nop_mse(_p(pred.cuda()), _p(tgt.cuda()), _p(wch.cuda()), 5, _p(grad), _p(loss), n, None) == 0
    lw = (wfull * (pred - tgt) ** 2).mean().item()
    assert abs(loss.item() - lw) <= 1e-5 * lw
    _close(grad.cpu(), 2 * wfull * (pred - tgt) / n, 8e-3)
    assert lib.clb_nop_mse(_p(pred.cuda()), _p(tgt.cuda()), None, 3, _p(grad), _p(loss), n - 1, None) == -1

    w, gr = torch.randn(n, generator=g), torch.randn(n, generator=g)
    wr = w.clone().requires_grad_(True)
    opt = torch.optim.Adam([wr], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    wd, m, v = w.cuda(), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    wb = torch.empty(n, device="cuda", dtype=torch.bfloat16)
    gd = gr.cuda()
    for t in range(1, 4):
        wr.grad = gr.clone()
        opt.step()
        assert lib.clb_nop_adam(_p(wd), _p(gd), _p(m), _p(v), _p(wb), n, 1e-2, 0.9, 0.999, 1e-8, t, None) == 0
    _close(wd.cpu(), wr.detach(), 1e-6)
    assert torch.equal(wb.cpu(), wd.cpu().to(torch.bfloat16))


def test_adam_multi_matches_the_single_tensor_step(lib):
    """Several tensors (more than one launch's 32) in one call: the same values
    as clb_nop_adam one tensor at a time, and the transposed BF16 copy."""
    from paper_2110_05943_gb300 import surrogate
    g = torch.Generator().manual_seed(23)
    shapes = [(216, 24), (1, 24), (72, 5), (1, 1)] * 9                     # 36 segments
    ts = []
    for r, c in shapes:
        w, gr = torch.randn((r, c), generator=g).cuda(), torch.randn((r, c), generator=g).cuda()
        ts.append(dict(r=r, c=c, w=w, g=gr, m=torch.zeros_like(w), v=torch.zeros_like(w),
                       wb=torch.empty((r, c), device="cuda", dtype=torch.bfloat16),
                       wbt=torch.empty((c, r), device="cuda", dtype=torch.bfloat16),
                       w1=w.clone(), m1=torch.zeros_like(w), v1=torch.zeros_like(w)))
    segs = (surrogate.AdamSeg * len(ts))(*[surrogate.AdamSeg(_p(q["w"]), _p(q["g"]), _p(q["m"]), _p(q["v"]), _p(q["wb"]),
                                                             _p(q["wbt"]), q["r"] * q["c"], q["r"], q["c"]) for q in ts])
    for t in range(1, 4):
        assert lib.clb_nop_adam_multi(segs, len(ts), 1e-2, 0.9, 0.999, 1e-8, t, None) == 0
        for q in ts:
            assert lib.clb_nop_adam(_p(q["w1"]), _p(q["g"]), _p(q["m1"]), _p(q["v1"]), None, q["r"] * q["c"], 1e-2, 0.9,
                                    0.999, 1e-8, t, None) == 0
    for q in ts:
        assert torch.equal(q["w"], q["w1"]) and torch.equal(q["m"], q["m1"]) and torch.equal(q["v"], q["v1"])
        assert torch.equal(q["wb"], q["w"].to(torch.bfloat16))
        assert torch.equal(q["wbt"], q["wb"].t())


class _RefNet(torch.nn.Module):
    """The surrogate's architecture in plain PyTorch FP32 with its real
    (unpadded) channel counts, the real parts of the weights copied in."""

    def __init__(self, net):
        super().__init__()
        self.w = [torch.nn.Parameter(l.real(l.wb).float().cpu().clone()) for l in net.layers]
        self.b = [torch.nn.Parameter(l.b[:l.cout_real].cpu().clone()) for l in net.layers]
        self.spec = [(l.cin_real, l.cout_real, l.taps, l.relu) for l in net.layers]

    def conv(self, i, x):
        cin, cout, taps, relu = self.spec[i]
        y = _ref_conv(x, self.w[i], taps, cin, cout, self.b[i])
        return y.clamp_min(0) if relu else y

    def forward(self, x):
        pool = lambda t: F.avg_pool2d(t.permute(0, 3, 1, 2), 2).permute(0, 2, 3, 1)
        up = lambda t: F.interpolate(t.permute(0, 3, 1, 2), scale_factor=2, mode="nearest").permute(0, 2, 3, 1)
        a2 = self.conv(1, self.conv(0, x))
        a4 = self.conv(3, self.conv(2, pool(a2)))
        a6 = self.conv(5, self.conv(4, pool(a4)))
        a8 = self.conv(7, self.conv(6, pool(a6)))
        a10 = self.conv(9, self.conv(8, torch.cat([up(a8), a6], dim=-1)))
        a12 = self.conv(11, self.conv(10, torch.cat([up(a10), a4], dim=-1)))
        a14 = self.conv(13, self.conv(12, torch.cat([up(a12), a2], dim=-1)))
        return self.conv(14, a14)


def _rel_l2(a, b):
    a, b = a.float().flatten(), b.float().flatten()
    return ((a - b).norm() / (b.norm() + 1e-30)).item()


def test_network_forward_backward_matches_autograd(lib):
    """One training step's output, loss gradient and every weight and bias
    gradient agree with PyTorch FP32 autograd of the same network to BF16
    activation accuracy (relative L2 error)."""
    from paper_2110_05943_gb300 import surrogate
    net = surrogate.Net.create(torch, seed=3)
    assert 1.0e6 < net.nparams < 1.3e6
    n, h, w = 2, 32, 24
    g = torch.Generator().manual_seed(21)
    x = torch.randn((n, h, w, surrogate.N_IN), generator=g).to(torch.bfloat16)
    y = torch.randn((n, h, w, 4), generator=g) * 0.3
    out, A = net.forward(x.cuda(), n, h, w)
    loss, dout = net.loss_and_grad(out, y.cuda())
    net.backward(dout, A, n, h, w)
    torch.cuda.synchronize()

    ref = _RefNet(net)
    o = ref(x.float())
    lref = F.mse_loss(o, y)
    lref.backward()
    assert _rel_l2(out.cpu(), o.detach()) < 2e-2
    assert abs(loss.item() / lref.item() - 1) < 2e-2
    for i, l in enumerate(net.layers):
        assert _rel_l2(l.real(l.gw).cpu(), ref.w[i].grad) < 6e-2, i
        assert _rel_l2(l.gb[:l.cout_real].cpu(), ref.b[i].grad) < 6e-2, i
        # the channel padding stays inert: its weights, biases and gradients are exactly zero
        gw = l.gw.clone().reshape(l.taps, l.cin, l.cout)
        gw[:, torch.as_tensor(l.rin, device=gw.device), :l.cout_real] = 0
        assert torch.count_nonzero(gw).item() == 0 and torch.count_nonzero(l.gb[l.cout_real:]).item() == 0, i
        wz = l.wb.float().clone().reshape(l.taps, l.cin, l.cout)
        wz[:, torch.as_tensor(l.rin, device=wz.device), :l.cout_real] = 0
        assert torch.count_nonzero(wz).item() == 0, i


def test_weights_round_trip_and_committed_weights_load(lib, tmp_path):
    """Saved weights are the real parts; loading them into a fresh (padded)
    network restores the same function.  The committed warm-start weights
    load into the current network."""
    import os
    from paper_2110_05943_gb300 import surrogate
    a = surrogate.Net.create(torch, seed=7)
    path = str(tmp_path / "w.npz")
    a.scale_coef = np.arange(9.0)
    a.save(path)
    b = surrogate.Net.create(torch, seed=8).load(path)
    for la, lb in zip(a.layers, b.layers):   # the BF16 weights inference uses, and the biases
        assert torch.equal(la.real(la.wb), lb.real(lb.wb)) and torch.equal(la.b, lb.b)
        assert torch.equal(lb.w, lb.wb.float())
    x = _bf((2, 16, 16, surrogate.N_IN), 31).cuda()
    oa, _ = a.forward(x, 2, 16, 16)
    ob, _ = b.forward(x, 2, 16, 16)
    assert torch.equal(oa, ob)
    pkg = os.path.dirname(os.path.abspath(surrogate.__file__))
    c = surrogate.Net.create(torch, seed=0).load(os.path.join(pkg, "weights", "warmstart_128.npz"))
    assert c.scale_coef is not None and c.nparams == a.nparams


def test_training_reduces_the_loss(lib):
    """Forty Adam steps on a smooth synthetic target cut the loss severalfold."""
    from paper_2110_05943_gb300 import surrogate
    net = surrogate.Net.create(torch, seed=4)
    rng = np.random.default_rng(5)
    n, h, w = 8, 32, 32
    X = rng.standard_normal((n, h, w, surrogate.N_IN)).astype(np.float32)
    yy, xx = np.mgrid[0:h, 0:w] / h
    Y = np.stack([np.sin(np.pi * xx) * X[:, :1, :1, 1], np.cos(np.pi * yy) * X[:, :1, :1, 2],
                  xx + 0 * X[:, :1, :1, 0], yy * X[:, :1, :1, 3]], axis=-1).astype(np.float32)
    hist = surrogate.train(net, X, Y, epochs=40, batch=8, lr=2e-3)
    assert np.isfinite(hist[-1][0])
    assert hist[-1][0] < 0.25 * hist[0][0], (hist[0][0], hist[-1][0])


def test_bounded_wait_expires_and_reports_timeout(lib):
    """The tensor-core kernels' failure path, made to run: a CTA waits on an
    mbarrier that nothing arrives at, with a bound of about 1 ms; the wait
    expires, the CTA frees its TMEM and sets the flag, clb_nop_check reports
    CLB_NOP_ERR_TIMEOUT once and clears it, and the context stays usable --
    a convolution afterwards still matches the reference."""
    assert lib.clb_nop_check(None) == 0
    assert lib.clb_nop_wait_selftest(0, None) == -1                 # bound outside 1 .. 4e9
    assert lib.clb_nop_wait_selftest(2_000_000, None) == 0
    assert lib.clb_nop_check(None) == -3                            # CLB_NOP_ERR_TIMEOUT
    assert lib.clb_nop_check(None) == 0                             # reported once, then cleared
    n, h, w, cin, cout = 1, 16, 16, 24, 32
    x, wm = _bf((n, h, w, cin), 41), _bf((9 * cin, cout), 42, 1 / 15)
    xd, wd, wtd = x.cuda(), wm.cuda(), wm.t().contiguous().cuda()
    y = torch.empty((n, h, w, cout), device="cuda")
    assert lib.clb_nop_conv_fwd(_p(xd), _p(wd), _p(wtd), None, _p(y), 1, 0, n, h, w, cin, cout, 9, None) == 0
    assert lib.clb_nop_check(None) == 0
    _close(y.cpu(), _ref_conv(x, wm, 9, cin, cout), 1e-5)
