"""Training and evaluation of the learned sketch-precision selector.

Every step runs in libmrcqr's kernels (features, MLP forward/backward,
AdamW); this module only generates data, drives the training loop and
stores the weights.  Data: synthetic m x n FP64 matrices A = U diag(sigma)
V^T (spectra geometric, step-cliff, clustered, log-uniform; n uniform in
[32, 512]; kappa_2 log-uniform in [1, 1e16]), each labelled by running MRCQR without
escalation at FP16 and at FP32: label 0 if FP16 passes the 1e-13 judge,
1 if only FP32 does, 2 otherwise (FP64).

    python -m paper_2606_18411_gb300.selector train --count 20000 --heldout 2000 \\
        --out paper_2606_18411_gb300/selector_weights.bin
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import struct
import time

import numpy as np
import torch

from . import _lib, inputs
from . import mrcqr as M

NF = 16
SPECTRA = inputs.SPECTRA
DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.bin")


def num_params() -> int:
    return _lib.load().mrcqr_selector_num_params()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return torch.cuda.current_stream().cuda_stream


def features_of(A: torch.Tensor, seed: int = 0, out: torch.Tensor | None = None) -> torch.Tensor:
    """The 16 selector features of the FP16 sketch's R_s of A (device)."""
    m, n = A.shape
    Y = M.sketch(A, 2 * n, "fp16", seed=seed)
    Rs = M.sketch_qr(Y, "fp16")
    f = out if out is not None else torch.empty(NF, dtype=torch.float32, device=A.device)
    _lib.check(_lib.load().mrcqr_selector_features(m, n, Rs.data_ptr(), f.data_ptr(), _stream()),
               "mrcqr_selector_features")
    return f


def passes(A: torch.Tensor, prec: str, seed: int = 0) -> bool:
    m, n = A.shape
    Q = M.empty_colmajor(m, n, device=A.device)
    R = M.empty_colmajor(n, n, device=A.device)
    M.factor_ex(A, Q, R, prec=prec, seed=seed, escalate=False)
    return M.last_status()["status"] == "OK"


def make_dataset(count: int, m: int, seed0: int, n_range=(32, 512), verify_fp64_every: int = 20, device="cuda",
                 log_every: int = 0):
    """Features X (count x 16), labels y, and (n, kappa, spectrum) of each matrix."""
    rng = np.random.default_rng(seed0)
    X = torch.empty((count, NF), dtype=torch.float32, device=device)
    y = np.zeros(count, dtype=np.int32)
    meta = []
    monotone_violations = 0
    t0 = time.time()
    for i in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        kind = SPECTRA[int(rng.integers(len(SPECTRA)))]
        kappa = float(10.0 ** rng.uniform(0.0, 16.0))
        A = inputs.make_matrix_torch(m, n, kappa, kind=kind, seed=seed0 * 1000003 + i, device=device)
        features_of(A, seed=i, out=X[i])
        p16 = passes(A, "fp16", seed=i)
        p32 = True if p16 else passes(A, "fp32", seed=i)
        y[i] = 0 if p16 else (1 if p32 else 2)
        if verify_fp64_every and i % verify_fp64_every == 0:
            p64 = passes(A, "fp64", seed=i)
            if not p64 or (p16 and not passes(A, "fp32", seed=i)):
                monotone_violations += 1
        meta.append((n, kappa, kind))
        if log_every and (i + 1) % log_every == 0:
            print(f"  {i + 1}/{count} matrices, {time.time() - t0:.0f} s", flush=True)
    torch.cuda.synchronize()
    return X, torch.from_numpy(y).to(device), meta, monotone_violations


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal hidden layers, small output layer, zero biases."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((64, 16)) * math.sqrt(2.0 / 16)
    W2 = rng.standard_normal((64, 64)) * math.sqrt(2.0 / 64)
    W3 = rng.standard_normal((3, 64)) * 0.01
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3.ravel(), np.zeros(3)]).astype(
        np.float32)


class Trainer:
    """FP32 master weights, Adam moments and BF16 copies on the device."""

    def __init__(self, params: np.ndarray, mu, sd, device="cuda"):
        self.master = torch.from_numpy(np.asarray(params, np.float32)).to(device)
        self.mom = torch.zeros_like(self.master)
        self.var = torch.zeros_like(self.master)
        self.wbf16 = self.master.to(torch.bfloat16).view(torch.int16)
        self.mu = torch.as_tensor(mu, dtype=torch.float32, device=device)
        self.sd = torch.as_tensor(sd, dtype=torch.float32, device=device)
        self.step = 0

    def train_step(self, X, y, class_w, lr=3e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4, apply=True,
                   grad_out=None):
        loss = torch.zeros(1, dtype=torch.float32, device=X.device)
        if apply:
            self.step += 1
        _lib.check(_lib.load().mrcqr_mlp_train_step(
            X.shape[0], X.data_ptr(), y.data_ptr(), class_w.data_ptr(), self.mu.data_ptr(), self.sd.data_ptr(),
            self.master.data_ptr(), self.mom.data_ptr(), self.var.data_ptr(), self.wbf16.data_ptr(), lr, beta1,
            beta2, eps, wd, max(self.step, 1), int(apply), _ptr(grad_out), loss.data_ptr(), _stream()),
            "mrcqr_mlp_train_step")
        return loss

    def forward(self, X, costs):
        logits = torch.empty((X.shape[0], 3), dtype=torch.float32, device=X.device)
        choice = torch.empty(X.shape[0], dtype=torch.int32, device=X.device)
        c = torch.as_tensor(costs, dtype=torch.float32, device=X.device)
        _lib.check(_lib.load().mrcqr_mlp_forward(X.shape[0], X.data_ptr(), self.wbf16.data_ptr(), self.mu.data_ptr(),
                                                 self.sd.data_ptr(), c.data_ptr(), logits.data_ptr(),
                                                 choice.data_ptr(), _stream()), "mrcqr_mlp_forward")
        return logits, choice


def train(X, y, epochs=40, batch=256, lr=3e-3, class_w=(1.0, 1.0, 2.0), seed=0, log=None):
    """Minibatch training; returns (trainer, mu, sd, losses per epoch)."""
    mu = X.mean(0).cpu().numpy()
    sd = X.std(0).cpu().numpy()
    sd[sd < 1e-6] = 1.0
    tr = Trainer(init_params(seed), mu, sd, device=X.device)
    cw = torch.tensor(class_w, dtype=torch.float32, device=X.device)
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    losses = []
    n = X.shape[0]
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        tot = 0.0
        for b in range(0, n, batch):
            idx = perm[b:b + batch]
            tot += float(tr.train_step(X[idx].contiguous(), y[idx].contiguous(), cw, lr=lr).item()) * len(idx)
        losses.append(tot / n)
        if log:
            log(f"epoch {ep + 1}: loss {losses[-1]:.4f}")
    return tr, mu, sd, losses


def save_weights(path, params, mu, sd, costs):
    with open(path, "wb") as f:
        f.write(b"MRCQRSEL")
        f.write(struct.pack("<II", 1, len(params)))
        f.write(np.asarray(mu, "<f4").tobytes())
        f.write(np.asarray(sd, "<f4").tobytes())
        f.write(np.asarray(costs, "<f4").tobytes())
        f.write(np.asarray(params, "<f4").tobytes())


def load_into_library(path: str = DEFAULT_WEIGHTS) -> None:
    _lib.check(_lib.load().mrcqr_selector_load(path.encode()), "mrcqr_selector_load")
    M._selector_state["loaded"] = True


def set_weights(params, mu, sd, costs) -> None:
    """Install weights held in memory (FP32 arrays) into the library."""
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (params, mu, sd, costs)]
    _lib.check(_lib.load().mrcqr_selector_set(*[a.ctypes.data for a in arrs]), "mrcqr_selector_set")
    M._selector_state["loaded"] = True


def measure_costs(m=1 << 16, n=256, reps=5, device="cuda"):
    """Relative time of one MRCQR run per sketch precision (FP16 = 1)."""
    A = inputs.make_matrix_torch(m, n, 10.0, seed=1, device=device)
    Q = M.empty_colmajor(m, n, device=device)
    R = M.empty_colmajor(n, n, device=device)
    t = []
    for p in ("fp16", "fp32", "fp64"):
        M.factor_ex(A, Q, R, prec=p, escalate=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            M.factor_ex(A, Q, R, prec=p, escalate=False)
        e1.record()
        torch.cuda.synchronize()
        t.append(e0.elapsed_time(e1) / reps)
    return [x / t[0] for x in t], t


def ladder_cost(start: int, label: int, costs) -> float:
    return costs[start] if start >= label else float(sum(costs[start:label + 1]))


def heldout_matrices(count: int, m: int, seed0: int = 2, n_range=(32, 512), device="cuda"):
    """The matrices of ``make_dataset(count, m, seed0)`` in order (the same draws), with (n, kappa, kind)."""
    rng = np.random.default_rng(seed0)
    for i in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        kind = SPECTRA[int(rng.integers(len(SPECTRA)))]
        kappa = float(10.0 ** rng.uniform(0.0, 16.0))
        yield i, inputs.make_matrix_torch(m, n, kappa, kind=kind, seed=seed0 * 1000003 + i, device=device), \
            (n, kappa, kind)


def evaluate_baselines(count: int, m: int, weights: str = DEFAULT_WEIGHTS, log_every: int = 0) -> dict:
    """The learned selector against the two estimators of Sec. II-C (the CholQR probe and the block
    1-norm estimate on A^T A) on the held-out set of ``train``: accuracy against the cheapest passing
    precision, under-predictions (each costs an escalation), and the cost of the precision ladder
    plus each estimator's own time, relative to the ideal choice (estimator time in units of one
    FP16-sketch run of the cost measurement)."""
    costs, times = measure_costs(m=m)
    load_into_library(weights)
    dev = "cuda"
    methods = ("learned", "probe", "onenorm")
    chosen = {k: [] for k in methods}
    est_ms = {k: 0.0 for k in methods}
    labels = []
    out = torch.empty(4, dtype=torch.float64, device=dev)
    stats = torch.zeros(8, dtype=torch.float64, device=dev)
    feat = torch.empty(NF, dtype=torch.float32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    for i, A, _ in heldout_matrices(count, m):
        mm, n = A.shape
        p16 = passes(A, "fp16", seed=i)
        p32 = True if p16 else passes(A, "fp32", seed=i)
        labels.append(0 if p16 else (1 if p32 else 2))
        # learned: the choice AUTO makes; its own cost is the FP16 sketch, its QR and the features
        e0.record()
        features_of(A, seed=i, out=feat)
        e1.record()
        torch.cuda.synchronize()
        est_ms["learned"] += e0.elapsed_time(e1)
        Q = M.empty_colmajor(mm, n, device=dev)
        R = M.empty_colmajor(n, n, device=dev)
        M.factor_ex(A, Q, R, prec="auto", seed=i, stats_device=stats)
        torch.cuda.synchronize()
        chosen["learned"].append(int(_lib.Stats.from_buffer_copy(stats.cpu().numpy().tobytes()).selector_choice))
        del Q, R
        for meth in ("probe", "onenorm"):
            e0.record()
            M.regime_estimate(A, meth, seed=i, out=out)
            e1.record()
            torch.cuda.synchronize()
            est_ms[meth] += e0.elapsed_time(e1)
            chosen[meth].append(int(out[1].item()))
        if log_every and (i + 1) % log_every == 0:
            print(f"  {i + 1}/{count} matrices, {time.time() - t0:.0f} s", flush=True)
    y = np.array(labels)
    ideal = sum(ladder_cost(int(l), int(l), costs) for l in y)
    rep = {"heldout_count": count, "m": m, "label_counts": np.bincount(y, minlength=3).tolist(),
           "relative_costs": costs, "run_ms": times,
           "always_fp32_relative_cost": sum(ladder_cost(1, int(l), costs) for l in y) / ideal,
           "always_fp64_relative_cost": sum(ladder_cost(2, int(l), costs) for l in y) / ideal, "methods": {}}
    for k in methods:
        c = np.array(chosen[k])
        conf = np.zeros((3, 3), dtype=int)
        for a, b in zip(y, c):
            conf[a, b] += 1
        ladder = sum(ladder_cost(int(ci), int(li), costs) for ci, li in zip(c, y))
        est_units = est_ms[k] / times[0]
        rep["methods"][k] = {"accuracy": float(np.mean(c == y)), "under_predictions": int(np.sum(c < y)),
                             "confusion_true_by_chosen": conf.tolist(),
                             "estimator_ms_mean": est_ms[k] / count,
                             "relative_cost_ladder": ladder / ideal,
                             "relative_cost_with_estimator": (ladder + est_units) / ideal}
    rep["seconds"] = time.time() - t0
    return rep


def policy_times(count: int, m: int, seed0: int = 5, n_choices=(64, 128, 256), reps: int = 2, device="cuda"):
    """Measured wall time of four policies over the same held-out mix (kappa_2 log-uniform in
    [1, 1e16], the four spectra, n from n_choices): AUTO (the selector's FP16 sketch, features and
    choice included), always FP16 and always FP32 (each escalating on failure) and always FP64.  Each matrix is factored
    once per policy per repetition, the policies interleaved per matrix; CUDA events around each
    call.  Returns total ms per policy and the statuses."""
    rng = np.random.default_rng(seed0)
    mats = []
    for i in range(count):
        n = int(rng.choice(n_choices))
        kind = SPECTRA[int(rng.integers(len(SPECTRA)))]
        kappa = float(10.0 ** rng.uniform(0.0, 16.0))
        mats.append((inputs.make_matrix_torch(m, n, kappa, kind=kind, seed=seed0 * 1000003 + i, device=device),
                     (n, kappa, kind)))
    load_into_library()
    tot = {"auto": 0.0, "fp16": 0.0, "fp32": 0.0, "fp64": 0.0}
    ok = {k: True for k in tot}
    stats = torch.zeros(8, dtype=torch.float64, device=device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for r in range(reps + 1):          # the first pass warms up
        for i, (A, _) in enumerate(mats):
            mm, n = A.shape
            Q = M.empty_colmajor(mm, n, device=device)
            R = M.empty_colmajor(n, n, device=device)
            for pol in ("auto", "fp16", "fp32", "fp64"):
                torch.cuda.synchronize()
                e0.record()
                M.factor_ex(A, Q, R, prec=pol, seed=i, stats_device=stats)
                e1.record()
                torch.cuda.synchronize()
                if r > 0:
                    tot[pol] += e0.elapsed_time(e1)
                    ok[pol] = ok[pol] and _lib.Stats.from_buffer_copy(stats.cpu().numpy().tobytes()).status == 0
    return {"count": count, "m": m, "n_choices": list(n_choices), "reps": reps,
            "total_ms": {k: v / reps for k, v in tot.items()}, "all_ok": ok,
            "auto_speedup": {"vs_fp16": tot["fp16"] / tot["auto"], "vs_fp32": tot["fp32"] / tot["auto"],
                             "vs_fp64": tot["fp64"] / tot["auto"]}}


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--count", type=int, default=20000)
    t.add_argument("--heldout", type=int, default=2000)
    t.add_argument("--m", type=int, default=1 << 16)
    t.add_argument("--epochs", type=int, default=40)
    t.add_argument("--n-max", type=int, default=512)
    t.add_argument("--cost-m", type=int, default=1 << 20, help="rows of the run-cost measurement")
    t.add_argument("--out", default=DEFAULT_WEIGHTS)
    t.add_argument("--report", default=None)
    b = sub.add_parser("baselines")
    b.add_argument("--heldout", type=int, default=2000)
    b.add_argument("--m", type=int, default=1 << 16)
    b.add_argument("--weights", default=DEFAULT_WEIGHTS)
    b.add_argument("--report", default=None)
    b.add_argument("--policy-count", type=int, default=48)
    b.add_argument("--policy-m", type=int, default=1 << 20)
    args = ap.parse_args()
    from . import build
    build.build()
    torch.cuda.set_device(0)
    if args.cmd == "baselines":
        rep = evaluate_baselines(args.heldout, args.m, args.weights, log_every=500)
        rep["measured_policy_times"] = policy_times(args.policy_count, args.policy_m)
        print(json.dumps(rep), flush=True)
        if args.report:
            with open(args.report, "w") as f:
                json.dump(rep, f, indent=1)
        return
    t0 = time.time()
    costs, times = measure_costs(m=args.cost_m)
    print(f"relative run costs fp16/fp32/fp64: {costs} ({times} ms)", flush=True)
    nr = (32, args.n_max)
    Xtr, ytr, _, v1 = make_dataset(args.count, args.m, seed0=1, n_range=nr, log_every=2000)
    Xte, yte, meta_te, v2 = make_dataset(args.heldout, args.m, seed0=2, n_range=nr, log_every=1000)
    t_data = time.time() - t0
    tr, mu, sd, losses = train(Xtr, ytr, epochs=args.epochs, log=lambda s: print(s, flush=True))
    params = tr.master.cpu().numpy()
    save_weights(args.out, params, mu, sd, costs)
    _, choice = tr.forward(Xte, costs)
    ch = choice.cpu().numpy()
    yt = yte.cpu().numpy()
    conf = np.zeros((3, 3), dtype=int)
    for a, b in zip(yt, ch):
        conf[a, b] += 1
    auto = sum(ladder_cost(int(c), int(l), costs) for c, l in zip(ch, yt))
    a32 = sum(ladder_cost(1, int(l), costs) for l in yt)
    a64 = sum(ladder_cost(2, int(l), costs) for l in yt)
    ideal = sum(ladder_cost(int(l), int(l), costs) for l in yt)
    rep = {"train_count": args.count, "heldout_count": args.heldout, "m": args.m, "cost_m": args.cost_m,
           "label_counts_train": np.bincount(ytr.cpu().numpy(), minlength=3).tolist(),
           "label_counts_heldout": np.bincount(yt, minlength=3).tolist(),
           "monotonicity_violations": int(v1 + v2), "relative_costs": costs, "run_ms": times,
           "final_train_loss": losses[-1], "heldout_accuracy": float(np.mean(ch == yt)),
           "confusion_true_by_chosen": conf.tolist(),
           "heldout_relative_cost": {"selector": auto / ideal, "always_fp32": a32 / ideal,
                                     "always_fp64": a64 / ideal, "ideal": 1.0},
           "under_predictions": int(np.sum(ch < yt)), "data_seconds": t_data,
           "total_seconds": time.time() - t0}
    print(json.dumps(rep), flush=True)
    if args.report:
        with open(args.report, "w") as f:
            json.dump(rep, f, indent=1)


if __name__ == "__main__":
    main()
