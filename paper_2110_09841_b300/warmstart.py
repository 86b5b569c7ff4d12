"""Learned warm start for CGLS: data, training and evaluation of the 3D U-Net.

Data: seeded random-ellipsoid phantoms on the CGLS geometry (128^3 @ 0.5 mm, 180 views /
360 deg, 256x192 detector @ 0.8 mm), projected by the CVP projector, with Poisson noise at
1e5 photons per pixel. Network input: the normalised backprojection A^T b / (A^T A 1);
target: the phantom. Evaluation: CGLS to the 1e-3 normal-equation residual from the network's
output x0 and from 0, on held-out seeds, in iterations and wall time (the warm start's time
includes the backprojection of b and the network's inference).

    python -m paper_2110_09841_b300.warmstart --train 2000 --epochs 3 --eval 100 --out result.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import torch

from . import inputs
from .kct import Projector
from .unet import UNet3D

TRAIN_SEED0 = 20000
EVAL_SEED0 = 10000
PHOTONS = 1e5


def phantom(geom, seed: int, device="cuda"):
    ph = inputs.WORKLOADS["cgls128"]["phantom"]
    edge = geom.nx * geom.ax
    return inputs.voxelize(geom, inputs.random_ellipsoids(seed, ph["count"], edge, ph["semi"], ph["mu"]),
                           device=device)


class Problem:
    """The operator of one geometry and the normalisation of its backprojection.

    The network input is A^T b / (A^T A 1): a constant volume c maps to c, so the input is a
    blurred estimate of the attenuation on the target's scale (A^T b / A^T 1 would instead be
    an average line integral, about 50 times the attenuation here)."""

    def __init__(self, geom, variant="relaxed"):
        self.geom = geom
        self.A = Projector(geom, variant, "cos")
        ones = torch.ones(geom.vol_shape, device="cuda")
        self.norm = self.A.backproject(self.A.project(ones))
        self.norm.clamp_(min=1e-6 * float(self.norm.max()))
        self.ws = self.A.cgls_workspace()

    def data(self, truth, seed: int):
        return inputs.poisson_log_data(self.A.project(truth), PHOTONS, seed)

    def network_input(self, b):
        return self.A.backproject(b) / self.norm


def generate(prob: Problem, seeds, target="phantom", tol=1e-3, max_iter=300):
    """(inputs, targets) float32 [N, nz, ny, nx] on the GPU. target "phantom": the phantom;
    "cgls": the CGLS solution from 0 at the stopping tolerance (what the warm start should
    reproduce so that few steps remain)."""
    g = prob.geom
    xs = torch.empty((len(seeds),) + g.vol_shape, device="cuda")
    ts = torch.empty_like(xs)
    for i, s in enumerate(seeds):
        t = phantom(g, s)
        b = prob.data(t, s)
        xs[i] = prob.network_input(b)
        if target == "cgls":
            prob.A.cgls(b, max_iter=max_iter, tol=tol, out=ts[i], workspace=prob.ws)
        else:
            ts[i] = t
    return xs, ts


def lr_factor(k: int, steps: int, warmup: int = 0) -> float:
    """Learning-rate factor of step k: a linear ramp over the first `warmup` steps, then a
    cosine from 1 down to 1/20 at step `steps` (held there afterwards)."""
    if k < warmup:
        return (k + 1) / warmup
    span = max(1, steps - warmup)
    k = min(k - warmup, span)
    return 0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * k / span))


def loss_value(out, target, edge_weight: float = 0.0):
    """Mean squared error of out [n, d, h, w], plus edge_weight times the mean squared error
    of its finite differences along each of the three axes. CGLS removes smooth errors of a
    start in few steps but sharp ones (a blurred edge) only slowly, so weighting the
    differences makes the start sharper where CGLS is slow."""
    e = out - target
    loss = torch.mean(e * e)
    if edge_weight > 0.0:
        for dim in (1, 2, 3):
            d = torch.diff(e, dim=dim)
            loss = loss + edge_weight * torch.mean(d * d)
    return loss


def train(model, xs, ts, epochs: int, lr: float = 1e-3, seed: int = 0, log=None, warmup: int = 0,
          clip: float = 0.0, log_every: int = 0, edge_weight: float = 0.0):
    """Adam on loss_value (the mean squared error, plus edge_weight times that of the finite
    differences), one volume per step, with the learning rate of lr_factor (optional linear
    warm-up, then a cosine from lr to lr / 20) and, if clip > 0, the gradient norm clipped to
    clip; the network's internal scale is set to 1 / mean |target|. Returns the mean loss of
    each epoch."""
    with torch.no_grad():
        model.scale.fill_(1.0 / float(ts.abs().mean().clamp(min=1e-12)))
    params = [p for p in model.parameters() if p.requires_grad]
    opt = torch.optim.Adam(params, lr=lr)
    steps = max(1, epochs * xs.shape[0])
    sched = torch.optim.lr_scheduler.LambdaLR(opt, lambda k: lr_factor(k, steps, warmup))
    gen = torch.Generator().manual_seed(seed)
    hist = []
    run, nrun, k = 0.0, 0, 0
    for ep in range(epochs):
        order = torch.randperm(xs.shape[0], generator=gen)
        tot = 0.0
        for i in order.tolist():
            opt.zero_grad(set_to_none=True)
            out = model(xs[i:i + 1])
            loss = loss_value(out, ts[i:i + 1], edge_weight)
            loss.backward()
            if clip > 0.0:
                torch.nn.utils.clip_grad_norm_(params, clip)
            opt.step()
            sched.step()
            value = float(loss.detach())
            tot += value
            run += value
            nrun += 1
            k += 1
            if log and log_every and k % log_every == 0:
                log(f"step {k}: mean loss of the last {nrun} steps {run / nrun:.3e}")
                run, nrun = 0.0, 0
        hist.append(tot / xs.shape[0])
        if log:
            log(f"epoch {ep}: mean loss {hist[-1]:.3e}")
    return hist


def evaluate(model, prob: Problem, seeds, tol=1e-3, max_iter=300):
    """Per seed: CGLS iterations and time from 0 and from the network's x0. The warm start's time
    counts the backprojection of b (the network input, which CGLS reuses as A^T b), the
    inference and CGLS from x0."""
    g = prob.geom
    rows = []
    x = torch.empty(g.vol_shape, device="cuda")
    for s in seeds:
        truth = phantom(g, s)
        b = prob.data(truth, s)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, cold = prob.A.cgls(b, max_iter=max_iter, tol=tol, out=x, workspace=prob.ws)
        torch.cuda.synchronize()
        t_cold = time.perf_counter() - t0
        err_cold = float((x - truth).norm() / truth.norm())
        t0 = time.perf_counter()
        atb = prob.A.backproject(b)             # the network input; CGLS reuses it as A^T b
        with torch.no_grad():
            x0 = model((atb / prob.norm)[None])[0].contiguous()
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - t0
        err_x0 = float((x0 - truth).norm() / truth.norm())
        _, warm = prob.A.cgls(b, x0=x0, max_iter=max_iter, tol=tol, out=x, workspace=prob.ws, atb=atb)
        torch.cuda.synchronize()
        t_warm = time.perf_counter() - t0
        rows.append({"seed": s, "iters_zero": cold["iterations"], "iters_warm": warm["iterations"],
                     "time_zero_s": t_cold, "time_warm_s": t_warm, "inference_s": t_inf,
                     "normal0_warm": float(warm["normal"][0]), "rel_err_x0": err_x0,
                     "rel_err_cgls_zero": err_cold, "rel_err_cgls_warm": float((x - truth).norm() / truth.norm()),
                     "converged": bool(cold["converged"] and warm["converged"])})
    return rows


def summarise(rows):
    def mean(k):
        return sum(r[k] for r in rows) / len(rows)

    return {k: mean(k) for k in ("iters_zero", "iters_warm", "time_zero_s", "time_warm_s", "inference_s",
                                 "normal0_warm", "rel_err_x0", "rel_err_cgls_zero", "rel_err_cgls_warm")} | {
        "seeds": len(rows), "all_converged": all(r["converged"] for r in rows),
        "warm_faster": sum(r["time_warm_s"] < r["time_zero_s"] for r in rows)}


def save_model(model, path: str):
    """Store the network's parameters and its input scale (FP32 master weights)."""
    torch.save({k: v.detach().cpu() for k, v in model.state_dict().items()}, path)


def load_model(model, path: str):
    """Load parameters and scale written by save_model into model (on the model's device)."""
    state = torch.load(path, map_location="cpu", weights_only=True)
    model.load_state_dict(state)
    return model


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--eval", type=int, default=100)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--warmup", type=int, default=0, help="steps of linear learning-rate warm-up")
    ap.add_argument("--clip", type=float, default=0.0, help="gradient-norm clipping (0: off)")
    ap.add_argument("--log-every", type=int, default=0, help="log the running loss every N steps")
    ap.add_argument("--edge-weight", type=float, default=0.0,
                    help="weight of the finite-difference term of the loss (0: plain mean squared error)")
    ap.add_argument("--variant", default="relaxed", choices=["exact", "relaxed"])
    ap.add_argument("--target", default="phantom", choices=["phantom", "cgls"])
    ap.add_argument("--out", default=None)
    ap.add_argument("--save", default=None, help="write the trained network's state to this file")
    ap.add_argument("--load", default=None, help="evaluate the network stored in this file instead of training")
    args = ap.parse_args()
    from . import build

    build.build()
    g = inputs.workload_geometry("cgls128")
    prob = Problem(g, args.variant)
    model = UNet3D().cuda()
    t_data = t_train = 0.0
    hist = []
    if args.load:
        load_model(model, args.load)
    else:
        t0 = time.perf_counter()
        xs, ts = generate(prob, range(TRAIN_SEED0, TRAIN_SEED0 + args.train), args.target)
        t_data = time.perf_counter() - t0
        t0 = time.perf_counter()
        hist = train(model, xs, ts, args.epochs, args.lr, log=print, warmup=args.warmup, clip=args.clip,
                     log_every=args.log_every, edge_weight=args.edge_weight)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        del xs, ts
    if args.save:
        save_model(model, args.save)
    rows = evaluate(model, prob, range(EVAL_SEED0, EVAL_SEED0 + args.eval))
    out = {"workload": "cgls128", "variant": args.variant, "target": args.target, "loaded": args.load,
           "train_samples": args.train,
           "epochs": args.epochs, "lr": args.lr, "warmup": args.warmup, "clip": args.clip,
           "edge_weight": args.edge_weight,
           "data_s": t_data, "train_s": t_train, "loss": hist, "summary": summarise(rows), "per_seed": rows}
    print(json.dumps(out["summary"]))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f)


if __name__ == "__main__":
    main()
