"""The learned rank predictor end to end: training data logged from the
full-SVD simulator, training by the library's GPU kernels, accuracy on
held-out updates, and what the trained predictor gains over the method
without it (the full Jacobi SVD) on a Loschmidt echo of weakly entangling
gates and on a Haar-random brickwork. On both, the rank a sketch must
capture (singular values above cutoff/100) is close to theta's smaller
dimension, so the predictor routes nearly every update to the full SVD: the
gain measured is about 1 (the predictor's cost against the sketches it
avoids). Every update is either sketched or routed; the results of both
runs agree within the binary64 tolerances; the predictor's overhead stays
bounded (gain above 0.8); the updates it routes to the full SVD are ones a
sketch could not have taken; the timings are printed."""
import time

import numpy as np
import pytest

from paper_1111_3124_gb300 import circuits as C
from tests.helpers import spectrum_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    t.cuda.set_device(0)
    from paper_1111_3124_gb300 import build as B
    B.build()
    from paper_1111_3124_gb300 import predictor as P
    X, T = P.training_set(seed=1, circuits=36)
    Xv, Tv = P.training_set(seed=2, circuits=8)
    p = P.train(X, T, seed=0, epochs=80)
    return P, p, (X, T), (Xv, Tv)


def test_predictor_learns_kept_rank(trained):
    P, p, (X, T), (Xv, Tv) = trained
    assert len(T) > 2000
    err = P.rank_error(p, Xv, Tv)
    print("held-out rank error:", err, "samples", len(T))
    assert err["median_rel"] < 0.25, err


def _timed(P, n, layers, chi, cutoff, pred):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m = P.run_with(n, layers, chi, cutoff, pred)
    m.sync()
    return m, time.perf_counter() - t0


@pytest.mark.parametrize("kind", ["echo", "haar"])
def test_gain_of_the_trained_predictor(trained, kind):
    P, p, _, _ = trained
    n, chi, cutoff, depth = 24, 128, 1e-10, 14
    rng = np.random.default_rng(77)
    layers = C.echo_brickwork(n, depth, rng, t_max=0.3) if kind == "echo" else C.brickwork(n, depth, rng)
    P.run_with(n, layers, chi, cutoff, None).sync()  # warm-up (workspace, modules)
    full, t_full = _timed(P, n, layers, chi, cutoff, None)
    skt, t_skt = _timed(P, n, layers, chi, cutoff, p)
    st = skt.sketch_stats()
    print(f"{kind}: full Jacobi {t_full:.3f} s, predictor+sketch {t_skt:.3f} s, gain x{t_full / t_skt:.2f}, {st}")
    for b in range(n - 1):
        assert spectrum_err(skt.schmidt(b), full.schmidt(b)) < 1e-12
    bits = np.random.default_rng(5).integers(0, 2, size=(32, n)).astype(np.uint8)
    assert np.max(np.abs(skt.amplitudes(bits) - full.amplitudes(bits))) < 1e-10
    assert st["sketched"] + st["routed_full"] == C.count_updates(layers)
    assert st["accepted"] <= st["sketched"]
    assert t_full / t_skt > 0.8, (t_full, t_skt)


def test_routing_quality_on_haar(trained):
    """Replayed on a full-SVD run (every update's true sketch rank known):
    what the predictor sends to the full SVD needed it, and what it would
    sketch would be accepted."""
    P, p, _, _ = trained
    n, chi, cutoff, depth = 24, 128, 1e-10, 14
    layers = C.brickwork(n, depth, np.random.default_rng(77))
    q = P.routing_quality(p, n, layers, chi, cutoff)
    print("routing quality:", q)
    assert q["sketched"] + q["routed_full"] == C.count_updates(layers)
    assert q["routed_full"] > 0 and q["full_needed"] >= 0.9, q
    if q["sketched"]:
        assert q["sketch_would_accept"] >= 0.8, q
