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
    if predictor is not None:
        m.set_predictor(predictor)
        m.set_mode(prec, 0, SVD_SKETCH_MLP)
    else:
        m.set_mode(prec, 0, SVD_JACOBI)
    m.run_layers(layers)
    return m
