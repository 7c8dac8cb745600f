"""The rank-predictor MLP's hand-written CUDA kernels against the binary64
CPU oracle (oracle/mlp.py), and the feature kernel against features computed
from the oracle's own state."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1111_3124_gb300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    t.cuda.set_device(0)
    from paper_1111_3124_gb300 import build as B
    B.build()
    from paper_1111_3124_gb300 import mps
    return mps


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, size=(n, 16)).astype(np.float32)
    T = (np.sin(X[:, 0] * 2) * 0.5 + X[:, 3] * X[:, 5] - 0.3 * X[:, 10]).astype(np.float32)
    return X, T


def test_forward_matches_oracle(lib):
    m = lib.RankPredictor(seed=3)
    X, _ = _data(100, 1)
    y_gpu = m.forward(X)
    y_ref, _ = mlp.forward(m.params.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(y_gpu - y_ref)) < 2e-5 * max(1.0, np.max(np.abs(y_ref)))


def test_backward_kernel_matches_oracle_gradient(lib):
    m = lib.RankPredictor(seed=4)
    X, T = _data(257, 2)
    loss, g = m.loss_grad(X, T)
    loss_ref, g_ref = mlp.loss_grad(m.params.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-5 * max(1.0, loss_ref)
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * max(1e-3, np.max(np.abs(g_ref)))


def test_training_on_gpu_reduces_loss(lib):
    m = lib.RankPredictor(seed=5)
    X, T = _data(4096, 3)
    l0, _ = m.loss_grad(X, T)
    l1 = m.train(X, T, epochs=40, batch=128, lr=3e-3, seed=1)
    l2, _ = m.loss_grad(X, T)
    assert l2 < 0.1 * l0, (l0, l1, l2)


def test_layer_features_match_oracle_state(lib):
    n, chi_max, cutoff = 10, 16, 1e-10
    layers = C.brickwork(n, 6, np.random.default_rng(8))
    ref = oracle.OracleMPS(n, chi_max, cutoff)
    for layer in layers:
        for s, U in layer:
            ref.apply_gate(s, U)
    g = lib.MPS(n, chi_max, cutoff)
    g.import_state(*ref.get_state()[1:])
    nxt = [(s, C.haar_unitary(4, np.random.default_rng(100 + s))) for s in C.brickwork_sites(n, 0)]
    X = g.layer_features([s for s, _ in nxt], np.stack([U for _, U in nxt]))
    chi, _, lams = ref.get_state()
    for row, (s, U) in zip(X, nxt):
        lam_l = lams[s - 1] if s >= 1 else np.ones(1)
        lam_r = lams[s + 1] if s + 1 <= n - 2 else np.ones(1)
        x = mlp.features(chi[s], chi[s + 1], chi[s + 2], mlp.entangling_power(U), lam_l, lam_r, cutoff)
        assert np.max(np.abs(row - x)) < 2e-6, (row, x)
