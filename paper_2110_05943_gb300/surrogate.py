"""Learned warm start for the porous-cavity time march.

A small convolutional neural operator (U-Net-like, four levels, ~1.1 M
parameters) maps the porosity field and (Ra, Da, Pr, sigma) of a cavity to
its steady (u, v, T) and density.  Its prediction initialises the LB time march
(clb_set_fields); the time march itself is unchanged, so the converged
answer is the solver's, and the plain cold start remains the fallback.

Every forward and backward pass runs in the library's kernels
(include/clb_nop.h): implicit-GEMM convolutions on the BF16 tensor cores
with FP32 accumulation, pooling, upsampling, concatenation, loss and Adam.
PyTorch only provides device memory and the stream.

Network (NHWC, BF16 activations, ReLU after every 3x3 convolution):
  enc1 128^2: 8 -> 24 -> 24        enc2 64^2: 24 -> 48 -> 48
  enc3 32^2: 48 -> 96 -> 96        bottom 16^2: 96 -> 192 -> 192
  dec3 32^2: [up 192 | 96] -> 96 -> 96
  dec2 64^2: [up 96 | 48] -> 48 -> 48
  dec1 128^2: [up 48 | 24] -> 24 -> 24       head: 1x1, 24 -> 4 (FP32)
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from . import clb

U_C = 0.1 / math.sqrt(3.0)     # characteristic velocity Ma c_s of Eq. 46, lattice units
# Boussinesq pressure variation across the cavity ~ g beta dT L = u_c^2, i.e.
# a density variation of ~3 u_c^2 = 0.01.
RHO_SCALE = 0.01
N_IN, N_OUT = 8, 4

_VP = ctypes.c_void_p


class AdamSeg(ctypes.Structure):
    """clb_nop_adam_seg of include/clb_nop.h."""
    _fields_ = [("w", _VP), ("g", _VP), ("m", _VP), ("v", _VP), ("wb", _VP), ("wbt", _VP), ("n", ctypes.c_int64),
                ("rows", ctypes.c_int32), ("cols", ctypes.c_int32)]


def _lib():
    L = clb.load()
    if not getattr(L, "_nop_ready", False):
        i32, i64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        L.clb_nop_conv_fwd.argtypes = [_VP, _VP, _VP, _VP, _VP, i32, i32, i32, i32, i32, i32, i32, i32, _VP]
        L.clb_nop_conv_dgrad.argtypes = [_VP, _VP, _VP, _VP, i32, i32, i32, i32, i32, i32, _VP]
        L.clb_nop_conv_wgrad.argtypes = [_VP, _VP, _VP, i32, i32, i32, i32, i32, i32, i32, _VP]
        L.clb_nop_conv_wgrad_bias.argtypes = [_VP, _VP, _VP, _VP, i32, i32, i32, i32, i32, i32, i32, _VP]
        L.clb_nop_bias_grad.argtypes = [_VP, _VP, i64, i32, _VP]
        L.clb_nop_pool2.argtypes = [_VP, _VP, i32, i32, i32, i32, i32, _VP]
        L.clb_nop_up2.argtypes = [_VP, _VP, i32, i32, i32, i32, i32, _VP]
        L.clb_nop_concat.argtypes = [_VP, _VP, _VP, i64, i32, i32, i32, _VP]
        L.clb_nop_mse.argtypes = [_VP, _VP, _VP, i32, _VP, _VP, i64, _VP]
        L.clb_nop_adam.argtypes = [_VP, _VP, _VP, _VP, _VP, i64, f32, f32, f32, f32, i32, _VP]
        L.clb_nop_adam_multi.argtypes = [ctypes.POINTER(AdamSeg), i32, f32, f32, f32, f32, i32, _VP]
        L.clb_nop_cast_bf16.argtypes = [_VP, _VP, i64, _VP]
        L.clb_nop_zero.argtypes = [_VP, i64, _VP]
        L.clb_nop_transpose.argtypes = [_VP, _VP, i32, i32, _VP]
        L.clb_nop_check.argtypes = [_VP]
        L.clb_nop_wait_selftest.argtypes = [i64, _VP]
        L.clb_nop_add_mask.argtypes = [_VP, _VP, _VP, _VP, i64, _VP]
        L._nop_ready = True
    return L


def _ok(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with status {rc}")


def _p(t):
    return None if t is None else t.data_ptr()


# ------------------------------------------------------------------ features
def features(phi: np.ndarray, Ra: float, Da: float, Pr: float, sigma: float) -> np.ndarray:
    """(H, W, 8) network input: normalised porosity, log10 Ra, log10 Da, Pr,
    sigma (broadcast), the two node coordinates and the mean porosity
    (broadcast).  Eight channels keep every layer's channel count a
    multiple of 8, the tensor-core path's granule."""
    phi = np.asarray(phi, dtype=np.float32)
    h, w = phi.shape
    out = np.empty((h, w, N_IN), dtype=np.float32)
    out[..., 0] = (phi - 0.65) / 0.15
    out[..., 1] = (math.log10(Ra) - 4.5) / 0.87
    out[..., 2] = (math.log10(Da) + 2.5) / 0.87
    out[..., 3] = (Pr - 0.85) / 0.087
    out[..., 4] = (sigma - 1.25) / 0.43
    out[..., 5] = np.linspace(-0.5, 0.5, w, dtype=np.float32)[None, :]
    out[..., 6] = np.linspace(-0.5, 0.5, h, dtype=np.float32)[:, None]
    out[..., 7] = (float(phi.mean()) - 0.65) / 0.15
    return out


def conduction_T(h: int, w: int, T_hot: float = 1.0, T_cold: float = 0.0) -> np.ndarray:
    """Pure-conduction temperature between the west (hot) and east (cold)
    wall nodes, x = 0 and x = w - 1: the Ra -> 0 limit of the cavity."""
    x = np.arange(w, dtype=np.float64) / (w - 1)
    return np.broadcast_to(T_hot + (T_cold - T_hot) * x, (h, w))


def _scale_terms(Ra, Da, Pr, sigma, eps_mean):
    a, d = math.log10(Ra), math.log10(Da)
    return np.array([1.0, a, d, math.log10(Pr), math.log10(sigma), eps_mean, a * a, d * d, a * d])


def fit_velocity_scale(params, u_rms):
    """Least-squares fit of log(u_rms / u_c) to a quadratic in (log10 Ra,
    log10 Da) plus linear terms in log10 Pr, log10 sigma and the mean
    porosity, over the training cases; params = [(Ra, Da, Pr, sigma, eps)]."""
    A = np.stack([_scale_terms(*p) for p in params])
    coef, *_ = np.linalg.lstsq(A, np.log(np.asarray(u_rms) / U_C), rcond=None)
    return coef


def velocity_scale(coef, Ra, Da, Pr, sigma, eps_mean) -> float:
    """Predicted RMS speed of the steady flow (lattice units)."""
    return float(U_C * math.exp(float(_scale_terms(Ra, Da, Pr, sigma, eps_mean) @ coef)))


def targets(rho: np.ndarray, ux: np.ndarray, uy: np.ndarray, T: np.ndarray, vscale: float) -> np.ndarray:
    """(H, W, 4) normalised steady fields: u / vscale, v / vscale,
    (T - T_conduction) / 0.5, (rho - mean rho) / RHO_SCALE.  Only density
    differences are learned: the walls' extrapolation leaks mass slowly, so
    the mean density of a converged run depends on its history."""
    Tc = conduction_T(*T.shape)
    return np.stack([ux / vscale, uy / vscale, (T - Tc) / 0.5, (rho - rho.mean()) / RHO_SCALE],
                    axis=-1).astype(np.float32)


def fields_from(pred: np.ndarray, vscale: float):
    """Inverse of targets(): (rho, ux, uy, T) in lattice units, mean density 1
    (the mass of the fluid at rest)."""
    pred = np.asarray(pred, dtype=np.float64)
    Tc = conduction_T(*pred.shape[:2])
    d = pred[..., 3] - pred[..., 3].mean()
    return (1.0 + RHO_SCALE * d, pred[..., 0] * vscale, pred[..., 1] * vscale, Tc + 0.5 * pred[..., 2])


def augment_rot180(X: np.ndarray, Y: np.ndarray):
    """Centro-symmetric copies of (features, targets).  With the hot wall at
    x = 0, the cold one at x = L, adiabatic top and bottom and buoyancy about
    T0 = (T_hot + T_cold) / 2, the Boussinesq Brinkman-Forchheimer equations
    map a solution (u, T, p)(x) on porosity eps(x) to (-u, 1 - T, p)(R x) on
    eps(R x), R the rotation by 180 degrees about the centre: velocities and
    the temperature deviation change sign, the pressure does not."""
    Xr = X.copy()
    Xr[..., 0] = X[:, ::-1, ::-1, 0]
    Yr = Y[:, ::-1, ::-1, :] * np.array([-1.0, -1.0, -1.0, 1.0], dtype=np.float32)
    return Xr, np.ascontiguousarray(Yr)


def peclet(vscale: float, nu: float, Pr: float, L: float) -> float:
    """Peclet number u L / alpha of the predicted flow (alpha = nu / Pr)."""
    return vscale * L * Pr / nu


# ------------------------------------------------------------------ layers
# Activations carry their channels padded with zeros to multiples of 32: the
# TMA-fed convolutions copy 32- or 64-channel boxes, and a box that runs past
# the last channel (24 of 32, say) is filled by the hardware at a large cost
# (a 24 -> 24 layer at 16 x 128^2 takes 55 us, a 32 -> 32 one 27 us).  The
# padding weights and biases are zero and stay zero (their gradients are
# exactly zero), so the padded network computes the same function as the
# real one; saved weights hold the real parts only.
def _pad32(c: int) -> int:
    return (c + 31) // 32 * 32


class Conv:
    """One convolution: FP32 master weights [taps * cin][cout] (cin, cout
    padded), BF16 copy and its transpose, FP32 bias, gradients and Adam
    moments.  rin: the padded positions of the real input channels;
    cout_real: the real outputs (the first ones)."""

    def __init__(self, torch, rin, cin, cout_real, taps, relu, rng, pad_out=True):
        self._torch = torch
        self.rin = np.asarray(list(rin), dtype=np.int64)
        self.cin_real, self.cout_real = len(self.rin), cout_real
        self.cin, self.cout, self.taps, self.relu = cin, (_pad32(cout_real) if pad_out else cout_real), taps, relu
        fan = taps * self.cin_real
        std = math.sqrt((2.0 if relu else 1.0) / fan)
        w = self.embed(rng.standard_normal((taps * self.cin_real, cout_real)).astype(np.float32) * std)
        dev = "cuda"
        self.w = torch.from_numpy(w).to(dev)
        self.wb = torch.empty(w.shape, dtype=torch.bfloat16, device=dev)
        self.b = torch.zeros(self.cout, dtype=torch.float32, device=dev)
        self.gw = torch.zeros_like(self.w)
        self.gb = torch.zeros_like(self.b)
        self.mw, self.vw = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.wbt = torch.empty((self.cout, taps * cin), dtype=torch.bfloat16, device=dev)   # for the forward
        _ok(_lib().clb_nop_cast_bf16(_p(self.w), _p(self.wb), self.w.numel(), None), "cast")
        self.refresh_t()

    def embed(self, real: np.ndarray) -> np.ndarray:
        """[taps * cin_real][cout_real] -> the padded [taps * cin][cout], zeros elsewhere."""
        out = np.zeros((self.taps, self.cin, self.cout), dtype=real.dtype)
        out[:, self.rin, :self.cout_real] = real.reshape(self.taps, self.cin_real, self.cout_real)
        return out.reshape(self.taps * self.cin, self.cout)

    def real(self, t):
        """The real part [taps * cin_real][cout_real] of a padded weight-shaped tensor."""
        idx = self._torch.as_tensor(self.rin, device=t.device)
        v = t.reshape(self.taps, self.cin, self.cout)[:, idx, :self.cout_real]
        return v.reshape(self.taps * self.cin_real, self.cout_real)

    def refresh_t(self):
        """Rebuild the transposed BF16 copy from the BF16 weights."""
        _ok(_lib().clb_nop_transpose(_p(self.wb), _p(self.wbt), self.taps * self.cin, self.cout, None), "transpose")

    @property
    def nparams(self):
        return self.taps * self.cin_real * self.cout_real + self.cout_real


@dataclass
class Net:
    layers: list
    torch: object
    scale_coef: object = None      # velocity-scale fit (fit_velocity_scale), stored with the weights

    @classmethod
    def create(cls, torch, seed=0, width=(24, 48, 96, 192), cin=N_IN, cout=N_OUT):
        rng = np.random.default_rng(seed)
        c1, c2, c3, c4 = width
        P = _pad32
        r = lambda c: range(c)
        cat = lambda a, b: list(range(a)) + [P(a) + j for j in range(b)]   # [up(a) | skip(b)], each padded
        spec = [(r(cin), P(cin), c1), (r(c1), P(c1), c1), (r(c1), P(c1), c2), (r(c2), P(c2), c2),
                (r(c2), P(c2), c3), (r(c3), P(c3), c3), (r(c3), P(c3), c4), (r(c4), P(c4), c4),
                (cat(c4, c3), P(c4) + P(c3), c3), (r(c3), P(c3), c3), (cat(c3, c2), P(c3) + P(c2), c2),
                (r(c2), P(c2), c2), (cat(c2, c1), P(c2) + P(c1), c1), (r(c1), P(c1), c1)]
        layers = [Conv(torch, ri, ci, co, 9, True, rng) for ri, ci, co in spec]
        layers.append(Conv(torch, r(c1), P(c1), cout, 1, False, rng, pad_out=False))
        net = cls(layers, torch)
        net.n_in = cin
        net._zeros = {}
        net._flat_grads()
        return net

    def _flat_grads(self):
        """All weight and bias gradients as views of one buffer (cleared by
        one call per backward pass), and the Adam segment table."""
        t = self.torch
        total = sum(l.gw.numel() + l.gb.numel() for l in self.layers)
        self.grads = t.zeros(total, dtype=t.float32, device="cuda")
        off = 0
        for l in self.layers:
            n = l.gw.numel()
            l.gw = self.grads[off:off + n].view(l.w.shape)
            off += n
            l.gb = self.grads[off:off + l.b.numel()]
            off += l.b.numel()
        segs = []
        for l in self.layers:
            segs.append(AdamSeg(_p(l.w), _p(l.gw), _p(l.mw), _p(l.vw), _p(l.wb), _p(l.wbt), l.w.numel(),
                                l.taps * l.cin, l.cout))
            segs.append(AdamSeg(_p(l.b), _p(l.gb), _p(l.mb), _p(l.vb), None, None, l.b.numel(), 1, l.b.numel()))
        self._segs = (AdamSeg * len(segs))(*segs)

    @property
    def nparams(self):
        return sum(l.nparams for l in self.layers)

    # resolution divisor of each layer (forward order)
    RES = (1, 1, 2, 2, 4, 4, 8, 8, 4, 4, 2, 2, 1, 1, 1)

    def train_flops(self, n, h, w):
        """Tensor-core FLOPs of one training step: forward, input gradient
        (all layers but the first) and weight gradient of every convolution."""
        tot = 0
        for i, (l, d) in enumerate(zip(self.layers, self.RES)):
            one = 2.0 * n * (h // d) * (w // d) * l.taps * l.cin_real * l.cout_real   # real channels
            tot += one * (2 if i == 0 else 3)
        return tot

    # ---- building blocks (all on the library's kernels)
    def _conv(self, l, x, n, h, w, out_f32=False):
        t = self.torch
        y = t.empty((n, h, w, l.cout), dtype=t.float32 if out_f32 else t.bfloat16, device="cuda")
        _ok(_lib().clb_nop_conv_fwd(_p(x), _p(l.wb), _p(l.wbt), _p(l.b), _p(y), int(out_f32), int(l.relu), n, h, w,
                                    l.cin, l.cout, l.taps, None), "conv_fwd")
        return y

    def _pool(self, x, n, h, w, c):
        y = self.torch.empty((n, h // 2, w // 2, c), dtype=self.torch.bfloat16, device="cuda")
        _ok(_lib().clb_nop_pool2(_p(x), _p(y), n, h, w, c, 0, None), "pool")
        return y

    def _up(self, x, n, h, w, c):
        y = self.torch.empty((n, 2 * h, 2 * w, c), dtype=self.torch.bfloat16, device="cuda")
        _ok(_lib().clb_nop_up2(_p(x), _p(y), n, h, w, c, 0, None), "up")
        return y

    def _cat(self, a, b, npix, ca, cb):
        y = self.torch.empty((npix, ca + cb), dtype=self.torch.bfloat16, device="cuda")
        _ok(_lib().clb_nop_concat(_p(a), _p(b), _p(y), npix, ca, cb, 0, None), "concat")
        return y

    def _pad_input(self, x, n, h, w):
        """(n, h, w, 8) -> (n, h, w, 32): the features and zero channels."""
        t, npix = self.torch, n * h * w
        pad = self.layers[0].cin - self.n_in
        z = self._zeros.get(npix)
        if z is None:
            z = self._zeros[npix] = t.zeros((npix, pad), dtype=t.bfloat16, device="cuda")
        y = t.empty((n, h, w, self.layers[0].cin), dtype=t.bfloat16, device="cuda")
        _ok(_lib().clb_nop_concat(_p(x), _p(z), _p(y), npix, self.n_in, pad, 0, None), "pad")
        return y

    def forward(self, x, n, h, w):
        """x: (n, h, w, 8) BF16 device tensor -> (n, h, w, 4) FP32, plus the
        activations the backward pass needs (channels padded to multiples of 32)."""
        L = self.layers
        c1, c2, c3, c4 = L[0].cout, L[2].cout, L[4].cout, L[6].cout
        x = self._pad_input(x, n, h, w)
        A = {"x": x}
        A[1] = self._conv(L[0], x, n, h, w)
        A[2] = self._conv(L[1], A[1], n, h, w)
        A["p1"] = self._pool(A[2], n, h, w, c1)
        A[3] = self._conv(L[2], A["p1"], n, h // 2, w // 2)
        A[4] = self._conv(L[3], A[3], n, h // 2, w // 2)
        A["p2"] = self._pool(A[4], n, h // 2, w // 2, c2)
        A[5] = self._conv(L[4], A["p2"], n, h // 4, w // 4)
        A[6] = self._conv(L[5], A[5], n, h // 4, w // 4)
        A["p3"] = self._pool(A[6], n, h // 4, w // 4, c3)
        A[7] = self._conv(L[6], A["p3"], n, h // 8, w // 8)
        A[8] = self._conv(L[7], A[7], n, h // 8, w // 8)
        A["u3"] = self._up(A[8], n, h // 8, w // 8, c4)
        A["c3"] = self._cat(A["u3"], A[6], n * (h // 4) * (w // 4), c4, c3)
        A[9] = self._conv(L[8], A["c3"], n, h // 4, w // 4)
        A[10] = self._conv(L[9], A[9], n, h // 4, w // 4)
        A["u2"] = self._up(A[10], n, h // 4, w // 4, c3)
        A["c2"] = self._cat(A["u2"], A[4], n * (h // 2) * (w // 2), c3, c2)
        A[11] = self._conv(L[10], A["c2"], n, h // 2, w // 2)
        A[12] = self._conv(L[11], A[11], n, h // 2, w // 2)
        A["u1"] = self._up(A[12], n, h // 2, w // 2, c2)
        A["c1"] = self._cat(A["u1"], A[2], n * h * w, c2, c1)
        A[13] = self._conv(L[12], A["c1"], n, h, w)
        A[14] = self._conv(L[13], A[13], n, h, w)
        out = self._conv(L[14], A[14], n, h, w, out_f32=True)
        return out, A

    # ---- backward
    def _grads(self, l, x, dy, n, h, w, mask, want_dx=True):
        """Accumulate l's weight and bias gradients; return dx (BF16) masked
        by `mask` > 0 (the ReLU of the layer that produced x) if given.  The
        weight gradient, which nothing before the optimiser step needs, runs
        on a side stream, overlapping the input-gradient chain of the
        default stream."""
        lib, t = _lib(), self.torch
        ev = t.cuda.Event()
        ev.record(t.cuda.default_stream())
        self._ws.wait_event(ev)
        _ok(lib.clb_nop_conv_wgrad_bias(_p(x), _p(dy), _p(l.gw), _p(l.gb), n, h, w, l.cin, l.cout, l.taps, 0,
                                        _VP(self._ws.cuda_stream)), "wgrad")
        x.record_stream(self._ws)
        dy.record_stream(self._ws)
        if not want_dx:
            return None
        dx = t.empty((n, h, w, l.cin), dtype=t.bfloat16, device="cuda")
        _ok(lib.clb_nop_conv_dgrad(_p(dy), _p(l.wb), _p(mask), _p(dx), n, h, w, l.cin, l.cout, l.taps, None),
            "dgrad")
        return dx

    def _split(self, y, npix, ca, cb):
        t = self.torch
        a = t.empty((npix, ca), dtype=t.bfloat16, device="cuda")
        b = t.empty((npix, cb), dtype=t.bfloat16, device="cuda")
        _ok(_lib().clb_nop_concat(_p(a), _p(b), _p(y), npix, ca, cb, 1, None), "split")
        return a, b

    def _add_mask(self, d1, d2, a):
        out = self.torch.empty_like(d1)
        _ok(_lib().clb_nop_add_mask(_p(d1), _p(d2), _p(a), _p(out), d1.numel(), None), "add_mask")
        return out

    def backward(self, dout, A, n, h, w):
        L, t, lib = self.layers, self.torch, _lib()
        c1, c2, c3, c4 = L[0].cout, L[2].cout, L[4].cout, L[6].cout
        if getattr(self, "_ws", None) is None:
            self._ws = t.cuda.Stream()
        _ok(lib.clb_nop_zero(_p(self.grads), self.grads.numel() * 4, None), "zero")
        h2, w2, h4, w4, h8, w8 = h // 2, w // 2, h // 4, w // 4, h // 8, w // 8
        d = self._grads(L[14], A[14], dout, n, h, w, A[14])
        d = self._grads(L[13], A[13], d, n, h, w, A[13])
        dc1 = self._grads(L[12], A["c1"], d, n, h, w, None)
        du1, d2_skip = self._split(dc1, n * h * w, c2, c1)
        d12 = t.empty((n, h2, w2, c2), dtype=t.bfloat16, device="cuda")
        _ok(lib.clb_nop_up2(_p(du1), _p(d12), n, h2, w2, c2, 1, None), "up_bwd")
        d = self._grads(L[11], A[11], self._add_mask(d12, None, A[12]), n, h2, w2, A[11])
        dc2 = self._grads(L[10], A["c2"], d, n, h2, w2, None)
        du2, d4_skip = self._split(dc2, n * h2 * w2, c3, c2)
        d10 = t.empty((n, h4, w4, c3), dtype=t.bfloat16, device="cuda")
        _ok(lib.clb_nop_up2(_p(du2), _p(d10), n, h4, w4, c3, 1, None), "up_bwd")
        d = self._grads(L[9], A[9], self._add_mask(d10, None, A[10]), n, h4, w4, A[9])
        dc3 = self._grads(L[8], A["c3"], d, n, h4, w4, None)
        du3, d6_skip = self._split(dc3, n * h4 * w4, c4, c3)
        d8 = t.empty((n, h8, w8, c4), dtype=t.bfloat16, device="cuda")
        _ok(lib.clb_nop_up2(_p(du3), _p(d8), n, h8, w8, c4, 1, None), "up_bwd")
        d = self._grads(L[7], A[7], self._add_mask(d8, None, A[8]), n, h8, w8, A[7])
        dp3 = self._grads(L[6], A["p3"], d, n, h8, w8, None)
        d6 = t.empty((n, h4, w4, c3), dtype=t.bfloat16, device="cuda")
        _ok(lib.clb_nop_pool2(_p(dp3), _p(d6), n, h4, w4, c3, 1, None), "pool_bwd")
        d = self._grads(L[5], A[5], self._add_mask(d6, d6_skip, A[6]), n, h4, w4, A[5])
        dp2 = self._grads(L[4], A["p2"], d, n, h4, w4, None)
        d4 = t.empty((n, h2, w2, c2), dtype=t.bfloat16, device="cuda")
        _ok(lib.clb_nop_pool2(_p(dp2), _p(d4), n, h2, w2, c2, 1, None), "pool_bwd")
        d = self._grads(L[3], A[3], self._add_mask(d4, d4_skip, A[4]), n, h2, w2, A[3])
        dp1 = self._grads(L[2], A["p1"], d, n, h2, w2, None)
        d2 = t.empty((n, h, w, c1), dtype=t.bfloat16, device="cuda")
        _ok(lib.clb_nop_pool2(_p(dp1), _p(d2), n, h, w, c1, 1, None), "pool_bwd")
        d = self._grads(L[1], A[1], self._add_mask(d2, d2_skip, A[2]), n, h, w, A[1])
        self._grads(L[0], A["x"], d, n, h, w, None, want_dx=False)
        done = t.cuda.Event()                 # the optimiser step waits for every weight gradient
        done.record(self._ws)
        t.cuda.default_stream().wait_event(done)

    def adam(self, step, lr, b1=0.9, b2=0.999, eps=1e-8):
        # one launch: every layer's weights (BF16 copy and its transpose refreshed) and biases
        _ok(_lib().clb_nop_adam_multi(self._segs, len(self._segs), lr, b1, b2, eps, step, None), "adam")

    def loss_and_grad(self, out, target, weights=None):
        """Channel-weighted MSE and its gradient (weights: device FP32, one per
        output channel, or None)."""
        t = self.torch
        loss = t.zeros(1, dtype=t.float32, device="cuda")
        g = t.empty(out.shape, dtype=t.bfloat16, device="cuda")
        _ok(_lib().clb_nop_mse(_p(out), _p(target), _p(weights), out.shape[-1], _p(g), _p(loss), out.numel(), None),
            "mse")
        return loss, g

    def state(self):
        """Real weights [taps * cin][cout] and biases of every layer (FP32)."""
        return [(l.real(l.w).cpu().numpy(), l.b[:l.cout_real].cpu().numpy()) for l in self.layers]

    def save(self, path):
        """Real weights as BF16 bit patterns (what inference uses) and FP32 biases."""
        arrs = {"scale_coef": np.asarray(self.scale_coef if self.scale_coef is not None else [], dtype=np.float64)}
        for i, l in enumerate(self.layers):
            arrs[f"w{i}"] = l.real(l.wb).contiguous().view(self.torch.int16).cpu().numpy()
            arrs[f"b{i}"] = l.b[:l.cout_real].cpu().numpy()
        np.savez_compressed(path, **arrs)

    def load(self, path):
        z = np.load(path)
        t = self.torch
        self.scale_coef = z["scale_coef"] if len(z["scale_coef"]) else None
        for i, l in enumerate(self.layers):
            real = (l.taps * l.cin_real, l.cout_real)
            if z[f"w{i}"].shape != real:
                raise ValueError(f"layer {i}: stored shape {z[f'w{i}'].shape} != {real}")
            wr = t.from_numpy(z[f"w{i}"]).view(t.bfloat16).float().numpy()
            l.w.copy_(t.from_numpy(l.embed(wr)).to("cuda"))     # BF16 values, exact in FP32
            _ok(_lib().clb_nop_cast_bf16(_p(l.w), _p(l.wb), l.w.numel(), None), "cast")
            l.b.zero_()
            l.b[:l.cout_real].copy_(t.from_numpy(z[f"b{i}"]).to("cuda"))
            l.refresh_t()
        return self


def to_bf16(torch, arr: np.ndarray):
    """Host FP32 array -> device BF16 tensor, converted by the library."""
    x = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float32)).to("cuda")
    y = torch.empty(x.shape, dtype=torch.bfloat16, device="cuda")
    _ok(_lib().clb_nop_cast_bf16(_p(x), _p(y), x.numel(), None), "cast")
    return y


def train(net: Net, X: np.ndarray, Y: np.ndarray, epochs: int, batch: int = 16, lr: float = 2e-3,
          Xval=None, Yval=None, log=None, weights=None):
    """Adam on the channel-weighted mean squared error (cosine learning-rate
    decay); X: (N, H, W, 8), Y: (N, H, W, 4).  Returns the per-epoch
    (train, validation) losses."""
    torch = net.torch
    n, h, w, _ = X.shape
    wd = None if weights is None else torch.tensor(weights, dtype=torch.float32, device="cuda")
    Xd = to_bf16(torch, X)
    Yd = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).to("cuda")
    hist = []
    step = 0
    rng = np.random.default_rng(1)
    nb = max(1, n // batch)
    total = epochs * nb
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).to("cuda")
        tot = 0.0
        for b in range(nb):
            idx = perm[b * batch:(b + 1) * batch]
            xb, yb = Xd.index_select(0, idx).contiguous(), Yd.index_select(0, idx).contiguous()
            out, A = net.forward(xb, xb.shape[0], h, w)
            loss, g = net.loss_and_grad(out, yb, wd)
            net.backward(g, A, xb.shape[0], h, w)
            step += 1
            cur = lr * 0.5 * (1.0 + math.cos(math.pi * step / total))
            net.adam(step, cur)
            tot += float(loss.item())
        val = evaluate(net, Xval, Yval, weights) if Xval is not None else None
        hist.append((tot / nb, val))
        if log:
            log(f"epoch {ep + 1}/{epochs}: train {tot / nb:.4e}" + (f"  val {val:.4e}" if val is not None else ""))
    return hist


def predict(net: Net, X: np.ndarray, batch: int = 16) -> np.ndarray:
    torch = net.torch
    n, h, w, _ = X.shape
    outs = []
    for b in range(0, n, batch):
        xb = to_bf16(torch, X[b:b + batch])
        out, _ = net.forward(xb, xb.shape[0], h, w)
        outs.append(out.cpu().numpy())
    return np.concatenate(outs, axis=0)


def warm_fields(net: Net, phi: np.ndarray, Ra: float, Da: float, Pr: float, sigma: float):
    """The network's steady (rho, ux, uy, T) for one cavity, in lattice
    units, ready for clb_set_fields."""
    X = features(phi, Ra, Da, Pr, sigma)[None]
    vs = velocity_scale(net.scale_coef, Ra, Da, Pr, sigma, float(np.mean(phi)))
    return fields_from(predict(net, X)[0], vs)


def evaluate(net: Net, X: np.ndarray, Y: np.ndarray, weights=None) -> float:
    """Channel-weighted mean squared error of the predictions."""
    P = predict(net, X)
    w = np.ones(Y.shape[-1]) if weights is None else np.asarray(weights, dtype=np.float64)
    return float(np.mean(np.mean((P - Y) ** 2, axis=(0, 1, 2)) * w))
