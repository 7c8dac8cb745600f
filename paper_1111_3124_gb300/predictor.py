"""Training data and training of the rank predictor (the learned part).

Samples are (features of a two-site update -> log2(r)/10) pairs logged from
runs of the full-SVD simulator (mps_layer_features before each layer,
mps_diag after it), where r is the rank a randomized sketch of the update
must capture to be accepted: the number of singular values above
max(cutoff/100, Mw eps) ||sigma|| (at least the kept rank). Training runs on the GPU by
the library's forward, backward and Adam kernels (mps_mlp_train).
"""
from __future__ import annotations

import numpy as np

from . import circuits as C
from .mps import MPS, PREC_FP64, SVD_JACOBI, SVD_SKETCH_MLP, RankPredictor


def collect(n: int, layers, chi_max: int, cutoff: float, prec: int = PREC_FP64):
    """Runs `layers` with the full Jacobi SVD and returns (X, T)."""
    m = MPS(n, chi_max, cutoff, prec)
    m.set_tuning(_tuning())
    Xs, Ts = [], []
    for layer in layers:
        one = [(s, U) for s, U in layer if U.shape[0] == 2]
        two = [(s, U) for s, U in layer if U.shape[0] == 4]
        if one:
            m.apply_layer([s for s, _ in one], np.stack([U for _, U in one]))
        if not two:
            continue
        sites = [s for s, _ in two]
        Us = np.stack([U for _, U in two])
        Xs.append(m.layer_features(sites, Us))
        m.apply_layer(sites, Us)
        Ts.append(np.log2(np.maximum(m.diag()["k_sketch"], 1)) / 10.0)
    m.close()
    if not Xs:
        return np.zeros((0, 16), np.float32), np.zeros(0, np.float32)
    return np.concatenate(Xs).astype(np.float32), np.concatenate(Ts).astype(np.float32)


def _tuning():
    from . import tuner
    return tuner.load() or []


def chi256_training_set(circuits: int, seed: int = 0, prec: int = 1):
    """Samples logged from circuits of the shape of the chi = 256 workload
    (n = 64, depth-20 Haar U(4) brickwork with RZ phases, chi_max = 256,
    cutoff 1e-12), 630 updates each, by the split-precision full SVD."""
    X, T = [], []
    for i in range(circuits):
        layers = C.brickwork(64, 20, np.random.default_rng(C.SEED_BASE + 50000 + 1000 * seed + i),
                             rz_after_each=True)
        x, t = collect(64, layers, 256, 1e-12, prec)
        X.append(x)
        T.append(t)
    return np.concatenate(X), np.concatenate(T)


def workload_mix(seed: int, count: int, n_range=(10, 33), chi_choices=(16, 32, 64, 128), depth_range=(6, 17)):
    """Mixed training circuits: Haar-random brickworks, weakly entangling
    brickworks and their Loschmidt echoes, of varied size, chi_max and cutoff."""
    rng = np.random.default_rng(seed)
    for i in range(count):
        n = int(rng.integers(*n_range))
        depth = int(rng.integers(*depth_range))
        chi = int(rng.choice(chi_choices))
        cutoff = float(rng.choice([1e-12, 1e-10, 1e-8]))
        crng = np.random.default_rng(seed * 1000 + i)
        if i % 3 == 0:
            layers = C.brickwork(n, depth, crng)
        elif i % 3 == 1:
            layers = C.weak_brickwork(n, depth, crng, t_max=float(rng.uniform(0.05, 0.4)))
        else:
            layers = C.echo_brickwork(n, depth // 2 + 1, crng, t_max=float(rng.uniform(0.05, 0.4)))
        yield n, layers, chi, cutoff


def training_set(seed: int = 0, circuits: int = 40, **kw):
    X, T = [], []
    for n, layers, chi, cutoff in workload_mix(seed, circuits, **kw):
        x, t = collect(n, layers, chi, cutoff)
        X.append(x)
        T.append(t)
    return np.concatenate(X), np.concatenate(T)


def train(X, T, seed: int = 0, epochs: int = 60, batch: int = 256, lr: float = 2e-3) -> RankPredictor:
    p = RankPredictor(seed=seed)
    p.train(X, T, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return p


def rank_error(p: RankPredictor, X, T) -> dict:
    """Prediction quality in rank units: median and 90th percentile of
    |predicted - r| / r, and the fraction under-predicted beyond the sketch's
    oversampling (which makes the sketch fall back)."""
    y = p.forward(X)
    kp, kt = np.exp2(10.0 * y), np.exp2(10.0 * T)
    rel = np.abs(kp - kt) / kt
    return {"median_rel": float(np.median(rel)), "p90_rel": float(np.quantile(rel, 0.9)),
            "under": float(np.mean(1.1 * kp + 10 < kt))}


def run_with(n, layers, chi_max, cutoff, predictor=None, prec: int = PREC_FP64):
    """Runs a circuit with the full Jacobi SVD (predictor None) or the
    predictor-sized sketch; returns the MPS."""
    m = MPS(n, chi_max, cutoff, prec)
    m.set_tuning(_tuning())
    if predictor is not None:
        m.set_predictor(predictor)
        m.set_mode(prec, 0, SVD_SKETCH_MLP)
    else:
        m.set_mode(prec, 0, SVD_JACOBI)
    m.run_layers(layers)
    return m


def routing_quality(predictor, n, layers, chi_max, cutoff, prec: int = PREC_FP64):
    """How the predictor would route each update of `layers` (replayed on a
    fresh full-SVD run, so every update's true sketch rank is known): the
    fraction of updates it sends to the sketch whose sketch would be accepted
    (true rank within the sketch's width), and the fraction it sends to the
    full SVD that did need it (true width 4r >= 3N)."""
    import math
    m = MPS(n, chi_max, cutoff, prec)
    m.set_tuning(_tuning())
    ok_s = n_s = ok_f = n_f = 0
    for layer in layers:
        one = [(s, U) for s, U in layer if U.shape[0] == 2]
        two = [(s, U) for s, U in layer if U.shape[0] == 4]
        if one:
            m.apply_layer([s for s, _ in one], np.stack([U for _, U in one]))
        if not two:
            continue
        sites = [s for s, _ in two]
        Us = np.stack([U for _, U in two])
        X = m.layer_features(sites, Us)
        chi = m.bond_dims()
        m.apply_layer(sites, Us)
        r_true = m.diag()["k_sketch"]
        r_hat = np.exp2(10.0 * np.clip(predictor.forward(X), -1.0, 1.1))
        for g, s in enumerate(sites):
            nw = min(2 * (chi[s - 1] if s > 0 else 1), 2 * (chi[s + 1] if s + 1 < n - 1 else 1))
            width = min(nw, math.ceil(1.1 * r_hat[g]) + 10)
            if 4 * width < 3 * nw and width < chi_max:
                n_s += 1
                ok_s += int(r_true[g] <= width)
            else:
                n_f += 1
                ok_f += int(4 * min(nw, r_true[g] + 10) >= 3 * nw or r_true[g] >= chi_max)
    m.close()
    return {"sketched": n_s, "sketch_would_accept": ok_s / max(n_s, 1), "routed_full": n_f,
            "full_needed": ok_f / max(n_f, 1)}


def deploy(predictor, n: int = 96, depth: int = 30, chi_max: int = 512, cutoff: float = 1e-10, prec: int = 1,
           seed: int = 0, kind: str = "haar"):
    """The deployment workload (Haar U(4) brickwork, or with kind "weak" a
    brickwork of weakly entangling gates exp(-it(XX+YY+ZZ)), t <= 0.15,
    dressed with Haar single-qubit gates; predictor-sized sketch with the full
    Jacobi SVD as fallback) against the full SVD on the same circuit: wall
    times, the gain, the sketch statistics, and the largest Schmidt-value and
    amplitude differences between the two runs."""
    import time
    import torch
    rng = np.random.default_rng(C.SEED_BASE + 5000 + seed)
    layers = C.brickwork(n, depth, rng) if kind == "haar" else C.weak_brickwork(n, depth, rng, t_max=0.15)
    out = {}
    runs = {}
    for name, pred in (("full", None), ("predictor", predictor)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = run_with(n, layers, chi_max, cutoff, pred, prec)
        m.sync()
        out[name + "_seconds"] = time.perf_counter() - t0
        runs[name] = m
    out["gain"] = out["full_seconds"] / out["predictor_seconds"]
    out.update(runs["predictor"].sketch_stats())
    out["updates"] = C.count_updates(layers)
    out["max_spectrum_diff"] = max(
        float(np.max(np.abs(runs["full"].schmidt(b) - runs["predictor"].schmidt(b))))
        if len(runs["full"].schmidt(b)) == len(runs["predictor"].schmidt(b)) else float("inf")
        for b in range(n - 1))
    bits = np.random.default_rng(1).integers(0, 2, size=(64, n)).astype(np.uint8)
    out["max_amp_diff"] = float(np.max(np.abs(runs["full"].amplitudes(bits) - runs["predictor"].amplitudes(bits))))
    out["max_bond"] = int(runs["full"].bond_dims().max())
    for m in runs.values():
        m.close()
    return out


def main() -> None:
    """python -m paper_1111_3124_gb300.predictor [--circuits 160] [--out PATH]
    [--deploy]: the chi = 256-shaped training set, training on the GPU,
    held-out accuracy, and (--deploy) the n = 96, chi_max = 512 deployment."""
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser()
    ap.add_argument("--circuits", type=int, default=160)
    ap.add_argument("--heldout", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--out", default=None)
    ap.add_argument("--deploy", action="store_true")
    ap.add_argument("--deploy-depth", type=int, default=30)
    ap.add_argument("--mix", type=int, default=0,
                    help="also train on this many mixed circuits (Haar, weak, echo; chi <= 128)")
    ap.add_argument("--deploy-weak", action="store_true")
    a = ap.parse_args()
    from . import build as B
    B.build()
    t0 = time.perf_counter()
    X, T = chi256_training_set(a.circuits, seed=1)
    Xv, Tv = chi256_training_set(a.heldout, seed=2)
    if a.mix:
        Xm, Tm = training_set(seed=3, circuits=a.mix)
        X, T = np.concatenate([X, Xm]), np.concatenate([T, Tm])
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    p = train(X, T, seed=0, epochs=a.epochs, batch=512, lr=2e-3)
    t_train = time.perf_counter() - t0
    rep = {"samples": int(len(T)), "heldout_samples": int(len(Tv)), "data_seconds": t_data,
           "train_seconds": t_train, "heldout": rank_error(p, Xv, Tv)}
    if a.out:
        np.save(a.out, p.params)
    if a.deploy:
        rep["deploy"] = deploy(p, depth=a.deploy_depth)
    if a.deploy_weak:
        rep["deploy_weak"] = deploy(p, depth=a.deploy_depth, kind="weak")
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
