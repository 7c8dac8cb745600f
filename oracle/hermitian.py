"""Plain CPU reference of the Hermitian-matrix workload of the paper's matrix
library (Sec. 2: diagonalisation of a Hermitian matrix; Sec. 2.1: exp_H, the
thermal state normalised by its trace, the pulse, the record of <X> under H,
zero padding and |DFT|).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and by ``bench.py``'s
reference legs. Every step is the definition written out with a library
routine where the definition names one: numpy's eigh for the eigenproblem,
scipy's Pade expm for the matrix exponential (an algorithm independent of the
eigenproblem), numpy's FFT for the DFT. A state evolves by exp(-i H t) for the
H given (pass 2 pi H for a Hamiltonian in Hz).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def heev(H):
    """Ascending eigenvalues and eigenvectors (columns) of a Hermitian matrix."""
    return np.linalg.eigh(np.asarray(H, dtype=np.complex128))


def expm(H, a: complex):
    """exp(a H) by scaling and squaring with a Pade approximant."""
    return scipy.linalg.expm(complex(a) * np.asarray(H, dtype=np.complex128))


def thermal(H, beta: float):
    """exp(-beta H) / Tr exp(-beta H) (Sec. 2.1, rho = exp_H(-beta H); rho /= trace)."""
    E = expm(H, -beta)
    return E / np.trace(E).real


def thermal_deviation(H, beta: float):
    """exp(-beta H) / Tr - I/D in H's eigenbasis, the weights written as
    (e_k - mean e) / (D (1 + mean e)) with e_k = expm1(-beta (lambda_k - lambda_0)),
    which is p_k - 1/D exactly and free of cancellation against 1/D."""
    w, V = heev(H)
    D = len(w)
    e = np.expm1(-beta * (w - w[0]))
    dev = (e - e.mean()) / (D * (1.0 + e.mean()))
    return (V * dev[None, :]) @ V.conj().T


def fid(rho, H, O, dt: float, ms, P=None):
    """Tr(exp(-i H t) rho' exp(i H t) O) at t = m dt for m in ms, rho' = P rho P^H."""
    rho = np.asarray(rho, dtype=np.complex128)
    if P is not None:
        P = np.asarray(P, dtype=np.complex128)
        rho = P @ rho @ P.conj().T
    out = np.zeros(len(ms), dtype=np.complex128)
    for i, m in enumerate(ms):
        U = expm(H, -1j * m * dt)
        out[i] = np.trace(U @ rho @ U.conj().T @ O)
    return out


def dft_abs(x, n_out: int):
    """|DFT| of x zero-padded to n_out values."""
    return np.abs(np.fft.fft(np.asarray(x, dtype=np.complex128), n_out))
