"""Brute-force state-vector simulator: the exhaustive O(2^n) representation
that Sec. 3.1 contrasts with the MPS form.

TEST INFRASTRUCTURE ONLY (pins the MPS oracle on n <= 14). psi is stored as an
n-axis tensor with axis q = qubit q; a gate's listed qubits are its index bits
from most to least significant (the convention fixed by the Sec. 3.2 example).
"""
from __future__ import annotations

import numpy as np


class StateVector:
    def __init__(self, n: int):
        self.n = n
        self.psi = np.zeros((2,) * n, dtype=np.complex128)
        self.psi[(0,) * n] = 1.0

    def apply(self, qubits, U) -> None:
        qubits = list(qubits)
        k = len(qubits)
        U = np.asarray(U, dtype=np.complex128).reshape((2,) * (2 * k))
        # out[i..., rest] = sum_{k...} U[i..., k...] psi[k..., rest]
        moved = np.moveaxis(self.psi, qubits, list(range(k)))
        out = np.tensordot(U, moved, axes=(list(range(k, 2 * k)), list(range(k))))
        self.psi = np.moveaxis(out, list(range(k)), qubits)

    def amplitude(self, bits) -> complex:
        return complex(self.psi[tuple(int(b) for b in bits)])

    def vector(self) -> np.ndarray:
        """Amplitudes indexed by the integer whose most significant bit is qubit 0."""
        return self.psi.reshape(-1).copy()

    def reduced_density(self, qubits) -> np.ndarray:
        qubits = list(qubits)
        k = len(qubits)
        rest = [q for q in range(self.n) if q not in qubits]
        m = np.moveaxis(self.psi, qubits + rest, list(range(self.n))).reshape(1 << k, -1)
        return m @ m.conj().T

    def expectation(self, qubits, O) -> complex:
        phi = StateVector(self.n)
        phi.psi = self.psi.copy()
        phi.apply(qubits, O)
        return complex(np.vdot(self.psi.reshape(-1), phi.psi.reshape(-1)))

    def schmidt(self, bond: int) -> np.ndarray:
        """Schmidt coefficients of the cut (0..bond)|(bond+1..n-1), Eq. (2),
        from the singular values of the reshaped amplitude vector."""
        m = self.psi.reshape(1 << (bond + 1), -1)
        return np.linalg.svd(m, compute_uv=False)
