"""Training and use of the seed network (learned initial pressure).

The network (built in the C library, ``osmodi_net_*``) maps the gradient
field and the mask to a pressure guess; training pairs are made by the
method itself: synthetic Gaussian-blob gradient fields solved by
``osmodi_solve`` to a tight tolerance.  A seeded solve runs the usual
iteration to the same tolerance from the network's guess and reports how far
the guess started (``seed_rel_dist``).
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import inputs
from . import osmodi as osm

# name, kind, cin, cout (the order of the library's parameter array)
LAYERS = [("e0", "conv3", 4, 16), ("e1", "down", 16, 32), ("e1b", "conv3", 32, 32), ("e2", "down", 32, 48),
          ("e2b", "conv3", 48, 48), ("e3", "down", 48, 64), ("m", "conv3", 64, 64), ("m2", "conv3", 64, 64),
          ("u2", "up", 64, 48), ("u2b", "conv3", 48, 48), ("u1", "up", 48, 32), ("u1b", "conv3", 32, 32),
          ("u0", "up", 32, 16), ("out", "conv1", 16, 1)]
TAPS = {"conv3": 27, "down": 8, "up": 8, "conv1": 1}


def init_params(seed=0) -> np.ndarray:
    """He-normal weights (taps, cin, cout) and zero biases, packed per layer."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, kind, cin, cout in LAYERS:
        taps = TAPS[kind]
        fan_in = cin * (taps if kind != "up" else 1)
        std = math.sqrt(2.0 / fan_in) if kind != "conv1" else math.sqrt(1.0 / fan_in)
        parts.append((rng.normal(size=(taps, cin, cout)) * std).ravel())
        parts.append(np.zeros(cout))
    return np.concatenate(parts).astype(np.float32)


def unpack(params: np.ndarray) -> dict:
    out = {}
    off = 0
    for name, kind, cin, cout in LAYERS:
        n = TAPS[kind] * cin * cout
        out[name + ".w"] = params[off:off + n].reshape(TAPS[kind], cin, cout)
        off += n
        out[name + ".b"] = params[off:off + cout]
        off += cout
    return out


def blob_problem(n, seed, device="cuda", noise=0.03):
    """The Gaussian-blob generator scaled to an n^3 box (widths 5-40 cells of
    a 500^3 box scaled by n/500, at least 1.5 cells)."""
    scale = n / 500.0
    lo, hi = max(1.5, 5.0 * scale), max(3.0, 40.0 * scale)
    return inputs.gaussian_blobs_3d(n=(n, n, n), noise=noise, seed=seed, width_range=(lo, hi), device=device,
                                    dtype=torch.float32)


def make_pairs(count, n, seed0=1000, tol=1e-8, device="cuda", precond=1):
    """Gradient fields and their converged pressures (targets)."""
    plan = osm.Plan(3, (n, n, n), (1.0, 1.0, 1.0), None, precision=osm.FP32_REFINE, precond=precond)
    pairs = []
    for i in range(count):
        prob = blob_problem(n, seed0 + i, device)
        p = torch.zeros((n, n, n), dtype=torch.float64, device=device)
        r = plan.solve(prob.grad, p, tol)
        if r.status != osm.OK:
            raise RuntimeError(f"target solve failed: {r.as_dict()}")
        pairs.append((prob.grad, p))
    plan.close()
    return pairs


def train(pairs, n, epochs=4, lr=1e-3, batch=4, seed=0, log=None, params=None):
    """Adam on the mean-removed MSE of the normalised pressure; returns the
    trained parameters and the loss history (per epoch)."""
    net = osm.Net((n, n, n), train=True)
    net.set_params(init_params(seed) if params is None else params)
    rng = np.random.default_rng(seed)
    hist = []
    k = 0
    for ep in range(epochs):
        order = rng.permutation(len(pairs))
        tot = 0.0
        for j, idx in enumerate(order):
            g, p = pairs[idx]
            tot += net.backward(g, None, 1.0, p, want_loss=True)
            k += 1
            if k % batch == 0:
                net.adam(lr, batch=batch)
        hist.append(tot / len(pairs))
        if log:
            log(f"epoch {ep} loss {hist[-1]:.5f}")
    out = net.get_params()
    net.close()
    return out, hist


def seeded_solve(params, grad, n, tol, plan=None, net=None):
    """P^0 from the network, then osmodi_solve to tol.  Returns (p, result,
    zero-start result) -- the zero-start solve of the same problem for
    comparison."""
    own_plan = plan is None
    own_net = net is None
    if own_plan:
        plan = osm.Plan(3, (n, n, n), (1.0, 1.0, 1.0), None, precision=osm.FP32_REFINE)
    if own_net:
        net = osm.Net((n, n, n), train=False)
        net.set_params(params)
    p = torch.empty((n, n, n), dtype=torch.float64, device=grad.device)
    net.forward(grad, None, 1.0, p)
    r_seed = plan.solve(grad, p, tol)
    p0 = torch.zeros_like(p)
    r_zero = plan.solve(grad, p0, tol)
    if own_plan:
        plan.close()
    if own_net:
        net.close()
    return p, r_seed, r_zero


def run_experiment(pairs=2000, train_n=128, epochs=4, lr=1e-3, batch=8, eval_n=256, eval_count=16, tol=1e-10,
                   log=print, params=None):
    """The network-seeded workload: train on `pairs` method-solved fields at
    train_n^3 (or take trained `params`), then solve `eval_count` held-out
    fields at eval_n^3 to `tol` from the network's guess and from zero, with
    the plain CG and with the multigrid-preconditioned CG.  Returns a result
    dict (and the parameters under "params")."""
    t_pairs = t_train = 0.0
    hist = []
    if params is None:
        t0 = time.perf_counter()
        data = make_pairs(pairs, train_n, tol=1e-8)
        torch.cuda.synchronize()
        t_pairs = time.perf_counter() - t0
        log(f"{pairs} training pairs at {train_n}^3 solved in {t_pairs:.1f} s")
        t1 = time.perf_counter()
        params, hist = train(data, train_n, epochs=epochs, lr=lr, batch=batch, log=log)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t1
        del data
        torch.cuda.empty_cache()
    plans = {"cg": osm.Plan(3, (eval_n,) * 3, (1.0, 1.0, 1.0), None, precision=osm.FP32_REFINE),
             "mg": osm.Plan(3, (eval_n,) * 3, (1.0, 1.0, 1.0), None, precision=osm.FP32_REFINE, precond=1)}
    # the plain FP64 solve (every vector and operation in FP64, same
    # preconditioned scheme, zero start): the time-to-tolerance reference
    plan64 = osm.Plan(3, (eval_n,) * 3, (1.0, 1.0, 1.0), None, precision=osm.FP64, precond=1)
    net = osm.Net((eval_n,) * 3, train=False)
    net.set_params(params)
    rows = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for i in range(eval_count):
        prob = blob_problem(eval_n, 50000 + i)
        row = dict(field=i)
        for name, plan in plans.items():
            p = torch.empty((eval_n,) * 3, dtype=torch.float64, device="cuda")
            plan.solve(prob.grad, torch.zeros_like(p), tol)  # warm (graph capture)
            ev[0].record()
            net.forward(prob.grad, None, 1.0, p)
            ev[1].record()
            r_seed = plan.solve(prob.grad, p, tol)
            ev[2].record()
            p0 = torch.zeros_like(p)
            r_zero = plan.solve(prob.grad, p0, tol)
            ev[3].record()
            torch.cuda.synchronize()
            row.update({f"{name}_seed_rel_dist": r_seed.seed_rel_dist, f"{name}_it_seeded": r_seed.inner_iters,
                        f"{name}_it_zero": r_zero.inner_iters, "ms_net": ev[0].elapsed_time(ev[1]),
                        f"{name}_ms_seeded_solve": ev[1].elapsed_time(ev[2]),
                        f"{name}_ms_zero_solve": ev[2].elapsed_time(ev[3]),
                        f"{name}_ok": r_seed.status == osm.OK and r_zero.status == osm.OK})
        p64 = torch.zeros((eval_n,) * 3, dtype=torch.float64, device="cuda")
        plan64.solve(prob.grad, p64, tol)  # warm
        p64.zero_()
        ev[0].record()
        r64 = plan64.solve(prob.grad, p64, tol)
        ev[1].record()
        torch.cuda.synchronize()
        row.update({"fp64_it_zero": r64.inner_iters, "fp64_ms_zero_solve": ev[0].elapsed_time(ev[1]),
                    "fp64_ok": r64.status == osm.OK})
        rows.append(row)
        log(str(rows[-1]))
    plan64.close()
    for plan in plans.values():
        plan.close()
    net.close()
    mean = lambda k: float(np.mean([r[k] for r in rows]))
    out = dict(pairs=pairs, train_n=train_n, epochs=epochs, lr=lr, batch=batch, eval_n=eval_n, eval_count=eval_count,
               tol=tol, seconds_pairs=t_pairs, seconds_train=t_train, loss_history=hist, ms_net=mean("ms_net"),
               all_converged=all(r["cg_ok"] and r["mg_ok"] and r["fp64_ok"] for r in rows), fields=rows,
               fp64=dict(mean_it_zero=mean("fp64_it_zero"), mean_ms_zero=mean("fp64_ms_zero_solve")))
    for name in plans:
        out[name] = dict(mean_seed_rel_dist=mean(f"{name}_seed_rel_dist"), mean_it_seeded=mean(f"{name}_it_seeded"),
                         mean_it_zero=mean(f"{name}_it_zero"),
                         mean_ms_seeded_total=mean("ms_net") + mean(f"{name}_ms_seeded_solve"),
                         mean_ms_zero=mean(f"{name}_ms_zero_solve"))
    out["params"] = [float(v) for v in np.asarray(params, dtype=np.float32)]
    return out


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description=run_experiment.__doc__)
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--train-n", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--eval-n", type=int, default=256)
    ap.add_argument("--eval-count", type=int, default=16)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--out", default=None)
    ap.add_argument("--params", default=None, help="JSON written by an earlier run: reuse its trained parameters")
    a = ap.parse_args()
    from . import build

    build.build()
    params = None
    if a.params:
        with open(a.params) as fh:
            params = np.asarray(json.load(fh)["params"], dtype=np.float32)
    res = run_experiment(a.pairs, a.train_n, a.epochs, a.lr, a.batch, a.eval_n, a.eval_count, a.tol, params=params)
    txt = json.dumps(res)
    print(json.dumps({k: v for k, v in res.items() if k not in ("fields", "params")}))
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(txt + "\n")
