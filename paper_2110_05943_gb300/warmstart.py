"""Learned warm start of the cavity time march, end to end.

1. Data: seeded 128^2 cavities (inputs.warmstart_cases: log10 Ra in [3, 6],
   log10 Da in [-4, -1], mean porosity in [0.4, 0.9] with a random porosity
   field, sigma in [0.5, 2], Pr in [0.7, 1]) advanced to steady state in one
   batched FP16-storage launch per step; a case retires when its hot-wall
   Nusselt number changes by at most `tol` (relative) over `every` steps.
2. Training: the surrogate network (surrogate.Net) on the first n_train
   cases, Adam on the mean squared error of the normalised fields.
   The training set is doubled by the cavity's centro-symmetry
   (surrogate.augment_rot180); the loss weighs the temperature most.
3. Evaluation on the held-out cases: the FP64 time march from rest (cold)
   and from the network's prediction (warm) until the relative residual
   (clb_residual over an interval of `check` steps) of both u and T is at
   most 1e-8; steps, wall time (network inference and upload included for
   the warm start), the step after which the hot-wall Nusselt number stays
   within 1e-4 of the cold run's converged value, and the final Nusselt
   numbers of both.

Run: python -m paper_2110_05943_gb300.warmstart --out <dir>
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import clb, surrogate
from .inputs import warmstart_cases


def _params(c, prec):
    return clb.clb_params_default(nx=c.nx, ny=c.ny, Ra=c.Ra, Da=c.Da, Pr=c.Pr, sigma=c.sigma, precision=prec)


def generate(cases, stream=None, tol=1e-5, every=4000, cap=400_000, log=None):
    """Steady (rho, ux, uy, T) of every case from the batched FP16N form.
    Returns (fields (N, 4, ny, nx) float32, steps per case, converged mask)."""
    n = len(cases)
    b = clb.Batch([_params(c, clb.CLB_F16N) for c, _ in cases], [phi for _, phi in cases],
                  [clb.clb_bc_cavity(1.0, 0.0) for _ in cases], stream=stream)
    b.tune(steps=3)
    active = np.ones(n, dtype=bool)
    steps = np.zeros(n, dtype=np.int64)
    prev = b.nusselt(clb.W)
    while active.any() and b.time < cap:
        b.step(every)
        cur = b.nusselt(clb.W)
        bad = active & ~np.isfinite(cur)
        done = active & np.isfinite(cur) & (np.abs(cur - prev) <= tol * np.abs(cur))
        steps[done | bad] = b.time
        active &= ~(done | bad)
        b.set_active(active)
        prev = cur
        if log:
            log(f"  t={b.time}: {int(active.sum())} active")
    steps[active] = b.time
    conv = ~active & np.isfinite(prev)
    out = np.empty((n, 4) + cases[0][1].shape, dtype=np.float32)
    for i in range(n):
        out[i] = np.stack(b.macros(i)).astype(np.float32)
    b.close()
    return out, steps, conv


def march(case, phi, init=None, stream=None, tol=1e-8, check=100, cap=600_000, nu_every=500, torch=None):
    """FP64 time march from rest (init None) or from init = (rho, ux, uy, T)
    until max(r_u, r_T) <= tol over `check`-step intervals.  Returns
    (steps, seconds, Nu_W, converged, Nu history [(t, Nu)] every nu_every)."""
    sim = clb.Simulation.create(_params(case, clb.CLB_F64), phi, clb.clb_bc_cavity(1.0, 0.0), stream=stream)
    try:
        if torch is not None:
            torch.cuda.synchronize()
        t0 = time.perf_counter()
        if init is not None:
            sim.set_fields(*init)
        sim.residual()
        hist = [(0, sim.nusselt(clb.W))]
        ok = False
        while sim.time < cap:
            sim.step(check)
            ru, rt = sim.residual()
            if sim.time % nu_every == 0:
                hist.append((sim.time, sim.nusselt(clb.W)))
            if max(ru, rt) <= tol:
                ok = True
                break
        nu = sim.nusselt(clb.W)
        hist.append((sim.time, nu))
        sec = time.perf_counter() - t0
        return sim.time, sec, nu, ok, hist
    finally:
        sim.close()


def steps_to_nu(hist, nu_ref, rel=1e-4):
    """First sampled time after which every sampled Nu stays within rel of
    nu_ref (None if the last sample is outside)."""
    t_ok = None
    for t, nu in hist:
        if abs(nu / nu_ref - 1.0) <= rel:
            if t_ok is None:
                t_ok = t
        else:
            t_ok = None
    return t_ok


LOSS_WEIGHTS = (1.0, 1.0, 2.0, 0.5)     # u, v, T, density: the temperature error costs the most steps


def run(out_dir, n_train=2000, n_test=200, epochs=120, batch=16, lr=2e-3, n_eval=None, seed=11, log=print):
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    res = {}
    cases = warmstart_cases(n_train + n_test, seed=seed)
    t0 = time.perf_counter()
    fields, steps, conv = generate(cases, stream=stream, log=log)
    res["data"] = {"cases": len(cases), "seconds": time.perf_counter() - t0, "converged": int(conv.sum()),
                   "steps_median": float(np.median(steps)), "steps_max": int(steps.max()),
                   "form": "FP16N batch, retire at |dNu| <= 1e-5 Nu per 4000 steps, cap 400000"}
    log(f"data: {res['data']}")
    good = conv & np.isfinite(fields).all(axis=(1, 2, 3))
    tr = [i for i in range(n_train) if good[i]]
    te = [i for i in range(n_train, n_train + n_test) if good[i]]
    u_rms = np.sqrt(np.mean(fields[:, 1].astype(np.float64) ** 2 + fields[:, 2].astype(np.float64) ** 2, axis=(1, 2)))
    prm = [(c.Ra, c.Da, c.Pr, c.sigma, float(np.mean(phi))) for c, phi in cases]
    net = surrogate.Net.create(torch, seed=0)
    net.scale_coef = surrogate.fit_velocity_scale([prm[i] for i in tr], u_rms[tr])
    vs = np.array([surrogate.velocity_scale(net.scale_coef, *p) for p in prm])
    res["params"] = net.nparams
    res["velocity_scale_fit"] = {"median_abs_log_error": float(np.median(np.abs(np.log(u_rms[te] / vs[te])))),
                                 "u_rms_range": [float(u_rms[tr].min()), float(u_rms[tr].max())]}
    X = np.stack([surrogate.features(phi, c.Ra, c.Da, c.Pr, c.sigma) for c, phi in cases])
    Y = np.stack([surrogate.targets(*fields[i].astype(np.float64), vs[i]) for i in range(len(cases))])
    Xr, Yr = surrogate.augment_rot180(X[tr], Y[tr])
    Xt, Yt = np.concatenate([X[tr], Xr]), np.concatenate([Y[tr], Yr])
    del Xr, Yr
    t0 = time.perf_counter()
    hist = surrogate.train(net, Xt, Yt, epochs=epochs, batch=batch, lr=lr, Xval=X[te], Yval=Y[te], log=log,
                           weights=LOSS_WEIGHTS)
    torch.cuda.synchronize()
    res["train"] = {"seconds": time.perf_counter() - t0, "epochs": epochs, "batch": batch, "lr": lr,
                    "train_cases": len(tr), "train_samples": len(Xt), "test_cases": len(te),
                    "augmentation": "rotation by 180 degrees (centro-symmetry)", "loss_weights": LOSS_WEIGHTS,
                    "loss_first": hist[0][0], "loss_last": hist[-1][0], "val_last": hist[-1][1]}
    del Xt, Yt
    net.save(os.path.join(out_dir, "warmstart_128.npz"))
    P = surrogate.predict(net, X[te])
    rel = {}
    for k, name in enumerate(("u", "v", "T", "rho")):
        num = np.sqrt(np.mean((P[..., k] - Y[te][..., k]) ** 2, axis=(1, 2)))
        den = np.sqrt(np.mean(Y[te][..., k] ** 2, axis=(1, 2))) + 1e-12
        rel[name] = float(np.median(num / den))
    Tabs = np.max(np.abs(P[..., 2] - Y[te][..., 2]) * 0.5, axis=(1, 2))
    res["test_field_error_median_rel_l2"] = rel
    res["test_T_max_abs_error_median"] = float(np.median(Tabs))
    log(f"train: {res['train']}  field error {rel}  T max abs (median) {np.median(Tabs):.3e}")

    ev = te if n_eval is None else te[:n_eval]
    rows = []
    for i in ev:
        c, phi = cases[i]
        ts = time.perf_counter()
        pred = surrogate.predict(net, X[i:i + 1])[0]
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - ts
        init = surrogate.fields_from(pred, vs[i])
        lat_nu = 0.1 * (c.ny - 1) * math.sqrt(c.Pr / (3.0 * c.Ra))       # Eq. 46, L = ny - 1
        pe = surrogate.peclet(vs[i], lat_nu, c.Pr, c.ny - 1)
        sc, tc, nc, okc, hc = march(c, phi, None, stream, torch=torch)
        sw, tw, nw, okw, hw = march(c, phi, init, stream, torch=torch)
        nc_t, nw_t = steps_to_nu(hc, nc), steps_to_nu(hw, nc)
        rows.append({"case": i, "Ra": c.Ra, "Da": c.Da, "Pr": c.Pr, "sigma": c.sigma, "eps_mean": c.phi,
                     "peclet_pred": pe,
                     "steps_cold": sc, "steps_warm": sw, "sec_cold": tc, "sec_warm": tw + t_inf,
                     "steps_nu_cold": nc_t, "steps_nu_warm": nw_t, "sec_inference": t_inf,
                     "nu_cold": nc, "nu_warm": nw, "rel_nu": abs(nw / nc - 1), "conv": bool(okc and okw)})
        log(f"  case {i} Pe {pe:.2f}: cold {sc} steps {tc:.2f}s  warm {sw} steps {tw + t_inf:.2f}s  "
            f"Nu-within-1e-4 at {nc_t} / {nw_t}  Nu {nc:.6f} / {nw:.6f}")
    conv_rows = [r for r in rows if r["conv"]]

    sc = np.array([r["steps_cold"] for r in conv_rows], float)
    sw = np.array([r["steps_warm"] for r in conv_rows], float)
    tc = np.array([r["sec_cold"] for r in conv_rows])
    tw = np.array([r["sec_warm"] for r in conv_rows])
    nc = np.array([r["steps_nu_cold"] or r["steps_cold"] for r in conv_rows], float)
    nw = np.array([r["steps_nu_warm"] or r["steps_warm"] for r in conv_rows], float)
    res["eval"] = {"cases": len(rows), "converged_both": len(conv_rows),
                   "criterion": "max(r_u, r_T) <= 1e-8 over 100-step intervals, FP64; and first step after which "
                                "Nu_W stays within 1e-4 of the cold run's converged Nu (500-step samples)",
                   "steps_cold_total": float(sc.sum()), "steps_warm_total": float(sw.sum()),
                   "sec_cold_total": float(tc.sum()), "sec_warm_total": float(tw.sum()),
                   "step_ratio_median": float(np.median(sw / sc)), "step_ratio_total": float(sw.sum() / sc.sum()),
                   "wall_speedup_total": float(tc.sum() / tw.sum()),
                   "nu_1e-4_steps_cold_total": float(nc.sum()), "nu_1e-4_steps_warm_total": float(nw.sum()),
                   "nu_1e-4_step_ratio_median": float(np.median(nw / nc)),
                   "warm_faster_cases": int(np.sum(sw < sc)),
                   "max_rel_nu": float(max(r["rel_nu"] for r in conv_rows)) if conv_rows else None}
    res["eval_rows"] = rows
    log(f"eval: {json.dumps(res['eval'], indent=1)}")
    with open(os.path.join(out_dir, "warmstart_128.json"), "w") as f:
        json.dump(res, f, indent=1)
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", default=".")
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=120)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--eval", type=int, default=None, help="held-out cases to time (default all)")
    a = ap.parse_args(argv)
    os.makedirs(a.out, exist_ok=True)
    run(a.out, a.train, a.test, a.epochs, a.batch, a.lr, a.eval)


if __name__ == "__main__":
    main()
