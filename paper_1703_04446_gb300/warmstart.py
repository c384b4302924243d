"""Learned warm start of the Gauss-Newton solve (an addition; the paper starts
every solve of Eq. 11 from zero or from a coarser level).

Pipeline, on one GPU, through the lgnk C ABI:
  1. pairs: T = random Gaussian blobs, v_true from the diffusion prior with at
     most 10 pixels of displacement (``synth.warmstart_pair``), R = u1(v_true, T)
     by the forward map (lgnk_forward);
  2. targets: v* = the zero-initialised Gauss-Newton solution of each training
     pair (lgnk_solve), i.e. the network learns what the solver returns;
  3. training: the lgnk_ws encoder-decoder (bf16 weights, FP32 accumulation,
     Adam with a cosine learning-rate decay) on (T, R) -> v*;
  4. evaluation on held-out pairs: Gauss-Newton from v = 0 with |g| <= 1e-3
     |g(0)| against Gauss-Newton from the prediction to the same absolute
     gradient norm.  The solver has the last word: when the prediction does not
     lower the objective below J(0), the solve starts from zero instead.

``python -m paper_1703_04446_gb300.warmstart`` runs the whole pipeline and
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import lgnk, synth

WORKLOAD = "2d_warmstart_128"
SCALE = 0.05            # network output scale: velocities are O(10 px) = O(0.08)
SOLVE = dict(max_gn=50, max_pcg=50, pcg_rtol=0.1)


def problem(**over):
    return lgnk.Problem.from_workload(synth.WORKLOADS[WORKLOAD], **over)


def make_pairs(ctx: lgnk.Context, first: int, count: int, seed: int = 0):
    """(T [n][128][128], R, v_true [n][1][2][64][64]) on the device."""
    wl = synth.WORKLOADS[WORKLOAD]
    m = wl.image.m[0]
    mv = wl.velocity.m[0]
    T = torch.empty((count, m, m), device=ctx.device)
    R = torch.empty_like(T)
    V = torch.empty((count, 1, 2, mv, mv), device=ctx.device)
    for k in range(count):
        t, v = synth.warmstart_pair(first + k, seed)
        T[k].copy_(torch.from_numpy(t))
        V[k].copy_(torch.from_numpy(v))
        R[k].copy_(ctx.forward(V[k], T[k]))
    return T, R, V


def solve_targets(ctx: lgnk.Context, T, R, rtol: float = 1e-3):
    """Zero-initialised Gauss-Newton solutions and their reports."""
    V = torch.empty((T.shape[0],) + tuple(ctx.problem.velocity_shape), device=ctx.device)
    reports = []
    for k in range(T.shape[0]):
        v, rep = ctx.solve(T[k], R[k], None, gn_grad_rtol=rtol, **SOLVE)
        V[k].copy_(v)
        reports.append(rep)
    return V, reports


def train(net: lgnk.WarmStart, T, R, V, epochs: int, batch: int, lr: float, seed: int = 0, lr_min: float = 1e-5):
    """Adam on minibatches of shuffled pairs; cosine decay from lr to lr_min.
    Returns the loss of every step."""
    n = T.shape[0]
    steps = epochs * (n // batch)
    rng = np.random.default_rng(seed)
    V2 = V.reshape(n, 2, V.shape[-2], V.shape[-1])
    losses, step = [], 0
    for _ in range(epochs):
        order = torch.from_numpy(rng.permutation(n)).to(T.device)
        for b in range(n // batch):
            idx = order[b * batch:(b + 1) * batch]
            rate = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * step / max(steps, 1)))
            losses.append(net.train_step(T[idx].contiguous(), R[idx].contiguous(), V2[idx].contiguous(), rate))
            step += 1
    return losses


def _sync():
    torch.cuda.synchronize()


def warm_solve(ctx: lgnk.Context, net: lgnk.WarmStart, T, R, rtol: float = 1e-3):
    """Gauss-Newton from the network's prediction to |g| <= rtol |g(0)|, the
    stopping point of the zero-initialised solve.  J(0) and g(0) are computed
    here (one objective-and-gradient call); when the prediction does not lower
    J below J(0) the solve starts from v = 0 instead.
    Returns (v, report, used_prediction, rtol |g(0)|)."""
    v0 = net.predict(T[None], R[None]).reshape(ctx.problem.velocity_shape)
    zero = torch.zeros_like(v0)
    J0, _, _, g = ctx.objective(zero, T, R, grad=True)
    gtol = rtol * math.sqrt(ctx.dot(g, g))
    Jp = ctx.objective(v0, T, R)[0]
    used = Jp < J0
    v, rep = ctx.solve(T, R, v0 if used else zero, gn_grad_rtol=0.0, gn_grad_atol=gtol, **SOLVE)
    return v, rep, used, gtol


def evaluate(ctx: lgnk.Context, net: lgnk.WarmStart, T, R, rtol: float = 1e-3):
    """Per held-out pair: zero-initialised solve to |g| <= rtol |g(0)|, then the
    warm-started solve to the same absolute gradient norm; wall times include
    the prediction and the J(0), J(v0) checks."""
    rows = []
    for k in range(T.shape[0]):
        _sync()
        t0 = time.perf_counter()
        vz, rz = ctx.solve(T[k], R[k], None, gn_grad_rtol=rtol, **SOLVE)
        _sync()
        t1 = time.perf_counter()
        vw, rw, used, _ = warm_solve(ctx, net, T[k], R[k], rtol)
        gtol = rtol * rz["g0"]
        _sync()
        t2 = time.perf_counter()
        rows.append(dict(zero_gn=rz["gn_iters"], zero_pcg=rz["pcg_iters"], zero_ms=1e3 * (t1 - t0),
                         zero_J=rz["J"], zero_ok=rz["g"] <= gtol * (1 + 1e-12),
                         warm_gn=rw["gn_iters"], warm_pcg=rw["pcg_iters"], warm_ms=1e3 * (t2 - t1),
                         warm_J=rw["J"], warm_ok=rw["g"] <= gtol * (1 + 1e-4), used=bool(used),
                         g0=rz["g0"], warm_g_start=rw["g0"]))
    return rows


def summarize(rows):
    def stat(key):
        a = np.array([r[key] for r in rows], dtype=np.float64)
        return {"mean": float(a.mean()), "median": float(np.median(a))}
    zt = sum(r["zero_ms"] for r in rows)
    wt = sum(r["warm_ms"] for r in rows)
    return {
        "pairs": len(rows),
        "zero": {"gn_iters": stat("zero_gn"), "pcg_iters": stat("zero_pcg"), "ms": stat("zero_ms"),
                 "converged": int(sum(r["zero_ok"] for r in rows))},
        "warm": {"gn_iters": stat("warm_gn"), "pcg_iters": stat("warm_pcg"), "ms": stat("warm_ms"),
                 "converged": int(sum(r["warm_ok"] for r in rows)),
                 "prediction_used": int(sum(r["used"] for r in rows))},
        "time_ratio_zero_over_warm": zt / wt if wt > 0 else None,
        "start_gradient_ratio": stat_ratio(rows),
        "final_J_ratio_warm_over_zero": float(np.median([r["warm_J"] / r["zero_J"] for r in rows])),
    }


def stat_ratio(rows):
    a = np.array([r["warm_g_start"] / r["g0"] for r in rows])
    return {"median": float(np.median(a)), "max": float(a.max())}


def forward_flops(m: int, c: int) -> float:
    """Multiply-adds x 2 of one forward pass on an m x m pair (the convolutions'
    logical work, without the padding the tensor-core tiles add)."""
    shapes = [(2, c, 1, 0, m), (c, 2 * c, 2, 0, m), (2 * c, 4 * c, 2, 0, m // 2), (4 * c, 8 * c, 2, 0, m // 4),
              (8 * c, 4 * c, 1, 1, m // 8), (4 * c, 2 * c, 1, 1, m // 4), (2 * c, 2, 1, 0, m // 2)]
    total = 0.0
    for ci, co, s, up, hin in shapes:
        ho = 2 * hin if up else hin // s
        total += 2.0 * ho * ho * co * ci * 9
    return total


def time_prediction(net: lgnk.WarmStart, T, R, reps: int = 50):
    """CUDA-event time of one prediction of one pair (ms)."""
    out = torch.empty((1, 2, T.shape[-1] // 2, T.shape[-1] // 2), device=T.device)
    for _ in range(3):
        net.predict(T[:1], R[:1], out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        net.predict(T[:1], R[:1], out=out)
    e1.record()
    _sync()
    return e0.elapsed_time(e1) / reps


def run(n_train=2048, n_test=256, channels=32, epochs=30, batch=32, lr=1e-3, seed=0, log=None, alpha=None):
    over = {} if alpha is None else {"alpha": alpha}
    ctx = lgnk.Context(problem(**over))
    out = {"workload": WORKLOAD, "alpha": ctx.problem.alpha, "train_pairs": n_train, "test_pairs": n_test,
           "base_channels": channels, "epochs": epochs, "batch": batch}
    t = time.perf_counter()
    T, R, _ = make_pairs(ctx, 0, n_train, seed)
    Tt, Rt, _ = make_pairs(ctx, 1_000_000, n_test, seed)
    _sync()
    out["pairs_s"] = time.perf_counter() - t
    t = time.perf_counter()
    V, reps = solve_targets(ctx, T, R)
    _sync()
    out["targets_s"] = time.perf_counter() - t
    out["targets_gn_iters_mean"] = float(np.mean([r["gn_iters"] for r in reps]))
    net = lgnk.WarmStart(T.shape[-1], channels, batch, SCALE)
    net.set_params(torch.from_numpy(synth.warmstart_init(channels, seed)))
    t = time.perf_counter()
    losses = train(net, T, R, V, epochs, batch, lr, seed)
    _sync()
    out["train_s"] = time.perf_counter() - t
    out["train_steps"] = len(losses)
    fl = forward_flops(T.shape[-1], channels)
    step_ms = 1e3 * out["train_s"] / max(len(losses), 1)
    out["train_step_ms"] = step_ms
    out["train_conv_tflops"] = 3.0 * fl * batch / (step_ms * 1e-3) / 1e12     # forward + two gradients
    pm = time_prediction(net, Tt, Rt)
    out["predict_ms"] = pm
    out["predict_conv_tflops"] = fl / (pm * 1e-3) / 1e12
    out["loss_first"], out["loss_last"] = losses[0], float(np.mean(losses[-20:]))
    rows = evaluate(ctx, net, Tt, Rt)
    out["eval"] = summarize(rows)
    if log:
        with open(log, "w") as f:
            json.dump({"summary": out, "rows": rows, "losses": losses}, f)
    net.close()
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--train", type=int, default=2048)
    ap.add_argument("--test", type=int, default=256)
    ap.add_argument("--channels", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--alpha", type=float, default=None, help="regularization weight (default: the workload's)")
    ap.add_argument("--log", default=None, help="JSON file for per-pair rows and losses")
    a = ap.parse_args()
    print(json.dumps(run(a.train, a.test, a.channels, a.epochs, a.batch, a.lr, a.seed, a.log, a.alpha)))


if __name__ == "__main__":
    main()
