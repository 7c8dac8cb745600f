"""CPU oracle of the rank-predictor MLP and of its gate feature e_p.

TEST INFRASTRUCTURE ONLY (imported by tests). binary64 throughout.

MLP: x (16) -> h = tanh(W1 x + b1) (64) -> y = w2 . h + b2; loss = mean (y - t)^2.
Parameter vector layout: W1[64][16], b1[64], w2[64], b2 (1153 values).

Entangling power (Zanardi, Zalka, Faoro, PRA 62, 030301, 2000): the mean,
over product inputs |a>|b> with |a>, |b> Haar-random, of the linear entropy
1 - Tr(rho_A^2) of U|a>|b>. The integrand is a polynomial of degree (2,2) in
(|a><a|, |b><b|), so the average over each qubit's six stabilizer states
(an octahedron, a spherical 3-design) is exact: a finite sum of 36 terms.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 16, 64
W1, B1 = 0, N_HID * N_IN
W2 = B1 + N_HID
B2 = W2 + N_HID
N_PARAMS = B2 + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return p[W1:B1].reshape(N_HID, N_IN), p[B1:W2], p[W2:B2], p[B2]


def forward(p, X):
    w1, b1, w2, b2 = unpack(p)
    H = np.tanh(np.asarray(X, dtype=np.float64) @ w1.T + b1)
    return H @ w2 + b2, H


def loss_grad(p, X, T):
    """Mean squared error and its gradient by backpropagation."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    w1, b1, w2, b2 = unpack(p)
    y, H = forward(p, X)
    B = len(T)
    r = y - T
    loss = float(np.mean(r ** 2))
    dy = 2.0 * r / B
    g = np.zeros(N_PARAMS)
    g[W2:B2] = H.T @ dy
    g[B2] = dy.sum()
    dz = np.outer(dy, w2) * (1.0 - H ** 2)
    g[B1:W2] = dz.sum(0)
    g[W1:B1] = (dz.T @ X).ravel()
    return loss, g


_STAB = [np.array(v, dtype=np.complex128) / np.linalg.norm(v) for v in
         ([1, 0], [0, 1], [1, 1], [1, -1], [1, 1j], [1, -1j])]


def entangling_power(U) -> float:
    U = np.asarray(U, dtype=np.complex128)
    acc = 0.0
    for a in _STAB:
        for b in _STAB:
            psi = (U @ np.kron(a, b)).reshape(2, 2)
            rho_a = psi @ psi.conj().T
            acc += 1.0 - float(np.real(np.trace(rho_a @ rho_a)))
    return acc / 36.0


def features(chi_l, chi_m, chi_r, ep, lam_l, lam_r, cutoff):
    """The 16 predictor features of a two-site gate (same definition as the
    product's feature kernel)."""
    pad = np.log(max(cutoff, 1e-13)) / 25.0
    x = [np.log2(chi_l) / 10.0, np.log2(chi_r) / 10.0, np.log2(chi_m) / 10.0, 4.5 * ep]
    for lam in (lam_l, lam_r):
        lam = np.sort(np.asarray(lam, dtype=np.float64))[::-1]
        x += [np.log(max(lam[i], 1e-30)) / 25.0 if i < len(lam) else pad for i in range(6)]
    return np.array(x)
