"""Pins for the MLP and entangling-power oracle (no GPU)."""
import numpy as np

from oracle import mlp
from paper_1111_3124_gb300 import circuits as C


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(0)
    p = rng.standard_normal(mlp.N_PARAMS) * 0.3
    X = rng.standard_normal((7, mlp.N_IN))
    T = rng.standard_normal(7)
    _, g = mlp.loss_grad(p, X, T)
    h = 1e-6
    idx = rng.choice(mlp.N_PARAMS, size=60, replace=False)
    idx = np.concatenate([idx, [mlp.B2, mlp.W2, mlp.B1, mlp.W1]])
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        fd = (mlp.loss_grad(p + e, X, T)[0] - mlp.loss_grad(p - e, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def test_entangling_power_closed_forms():
    assert abs(mlp.entangling_power(np.eye(4))) < 1e-15
    assert abs(mlp.entangling_power(C.SWAP)) < 1e-15
    assert abs(mlp.entangling_power(C.CNOT) - 2.0 / 9.0) < 1e-15  # the maximum for qubits
    rng = np.random.default_rng(1)
    for _ in range(5):
        U = C.haar_unitary(4, rng)
        ep = mlp.entangling_power(U)
        assert 0.0 <= ep <= 2.0 / 9.0 + 1e-15
        L = np.kron(C.haar_unitary(2, rng), C.haar_unitary(2, rng))
        R = np.kron(C.haar_unitary(2, rng), C.haar_unitary(2, rng))
        assert abs(mlp.entangling_power(L @ U @ R) - ep) < 1e-14  # local invariance


def test_entangling_power_is_haar_average():
    """The 3-design sum equals the Haar average (Monte Carlo, 4 sigma)."""
    rng = np.random.default_rng(2)
    U = C.haar_unitary(4, rng)
    vals = []
    for _ in range(20000):
        a = C.haar_unitary(2, rng)[:, 0]
        b = C.haar_unitary(2, rng)[:, 0]
        psi = (U @ np.kron(a, b)).reshape(2, 2)
        ra = psi @ psi.conj().T
        vals.append(1.0 - np.real(np.trace(ra @ ra)))
    vals = np.array(vals)
    assert abs(vals.mean() - mlp.entangling_power(U)) < 4 * vals.std() / np.sqrt(len(vals))
