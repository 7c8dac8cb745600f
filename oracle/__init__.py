"""Plain CPU oracle for the Vidal-form MPS gate update (Sec. 3.1, Eq. 1-2).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``. The product library never imports
it, and the two share no code.

``mps_oracle.cpp`` holds the arithmetic (binary64 and binary128 modes);
``statevector.py`` is an independent brute-force state-vector simulator used to
pin it. This module only compiles the C++ file and marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mps_oracle.cpp")
_LIB = os.path.join(_HERE, "libmps_oracle.so")
_lib = None

FP64 = 0
BINARY128 = 1


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (no GPU, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared",
                               "-fno-fast-math", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_mps_create.restype = P
        L.oracle_mps_create.argtypes = [I, I, D, I]
        L.oracle_mps_destroy.argtypes = [P]
        L.oracle_mps_apply_gate.argtypes = [P, I, I, dp]
        L.oracle_mps_amplitude.argtypes = [P, ctypes.c_char_p, dp]
        L.oracle_mps_expectation.argtypes = [P, I, I, dp, dp]
        L.oracle_mps_reduced_density.argtypes = [P, ip, I, dp]
        L.oracle_mps_bond_dim.argtypes = [P, I]
        L.oracle_mps_get_schmidt.argtypes = [P, I, dp]
        L.oracle_mps_set_state.argtypes = [P, ip, dp, dp]
        L.oracle_mps_get_state.argtypes = [P, ip, dp, dp]
        L.oracle_mps_last_diag.argtypes = [P, ip, dp, ip, ip]
        L.oracle_svd.argtypes = [I, I, I, dp, dp, dp, dp]
        L.oracle_mps_sample.argtypes = [P, dp, ctypes.c_char_p]
        L.oracle_mps_pauli.argtypes = [P, ctypes.c_char_p, dp]
        L.oracle_mps_apply_gate_hl.argtypes = [P, I, I, dp, dp]
        L.oracle_mps_amplitude_hl.argtypes = [P, ctypes.c_char_p, dp]
        L.oracle_mps_get_schmidt_hl.argtypes = [P, I, dp, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def svd(T, prec: int = FP64):
    """SVD of a complex matrix: returns (sigma, X, Y, sweeps) with T = X diag(sigma) Y^H.

    sigma is in Jacobi column order (not sorted)."""
    T = _c128(T)
    m, n = T.shape
    r = min(m, n)
    sigma = np.zeros(r)
    X = np.zeros((r, m), dtype=np.complex128)  # column-major m x r
    Y = np.zeros((r, n), dtype=np.complex128)
    sw = lib().oracle_svd(prec, m, n, _dp(T.view(np.float64)), _dp(sigma),
                          _dp(X.view(np.float64)), _dp(Y.view(np.float64)))
    return sigma, X.T.copy(), Y.T.copy(), sw


class OracleMPS:
    """Vidal-form MPS of n qubits, |0...0> at creation (Sec. 3.2 example)."""

    def __init__(self, n: int, chi_max: int, cutoff: float, prec: int = FP64):
        self.n, self.chi_max, self.cutoff, self.prec = n, chi_max, cutoff, prec
        self._h = lib().oracle_mps_create(n, chi_max, cutoff, prec)
        if not self._h:
            raise ValueError("bad oracle arguments")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_mps_destroy(h)
            self._h = None

    def apply_gate(self, site: int, U) -> None:
        U = _c128(U)
        k = {2: 1, 4: 2, 8: 3}[U.shape[0]]
        rc = lib().oracle_mps_apply_gate(self._h, site, k, _dp(U.view(np.float64)))
        if rc != 0:
            raise RuntimeError("oracle gate failed: %d" % rc)

    def apply_gate_hl(self, site: int, U_hi, U_lo=None) -> None:
        """Gate whose entries are hi + lo exactly (formed in the oracle's
        precision; lo may be None)."""
        hi = _c128(U_hi)
        k = {2: 1, 4: 2, 8: 3}[hi.shape[0]]
        lo = None if U_lo is None else _c128(U_lo)
        rc = lib().oracle_mps_apply_gate_hl(self._h, site, k, _dp(hi.view(np.float64)),
                                            None if lo is None else _dp(lo.view(np.float64)))
        if rc != 0:
            raise RuntimeError("oracle gate failed: %d" % rc)

    def amplitude_hl(self, bits) -> np.ndarray:
        """<bits|psi> as (re hi, re lo, im hi, im lo): in binary128 mode the
        value rounded to a pair of doubles."""
        b = bytes(bytearray(int(x) & 1 for x in bits))
        out = np.zeros(4)
        lib().oracle_mps_amplitude_hl(self._h, b, _dp(out))
        return out

    def schmidt_hl(self, b: int):
        """(hi, lo) of Lambda_b."""
        k = self.bond_dim(b)
        hi, lo = np.zeros(k), np.zeros(k)
        lib().oracle_mps_get_schmidt_hl(self._h, b, _dp(hi), _dp(lo))
        return hi, lo

    def apply_gate_on(self, qubits, U, route: str = "embed") -> None:
        """Gate on listed qubits (first = most significant). Adjacent increasing
        qubits go straight through; a two-qubit gate on (q, q+2) is embedded as
        an 8x8 gate on (q, q+1, q+2) with the identity on q+1 (route "embed");
        otherwise SWAP gates carry the higher qubit next to the lower one and
        back (route "swap", and every distance above 2)."""
        U = _c128(U)
        qubits = list(qubits)
        if len(qubits) == 1 or all(qubits[t + 1] == qubits[t] + 1 for t in range(len(qubits) - 1)):
            self.apply_gate(qubits[0], U)
            return
        if len(qubits) == 2 and (abs(qubits[1] - qubits[0]) > 2 or route == "swap" or qubits[1] == qubits[0] - 1):
            q0, q1 = qubits
            if q0 > q1:  # index bits in increasing qubit order
                P = np.zeros((4, 4))
                for a in range(2):
                    for b in range(2):
                        P[b * 2 + a, a * 2 + b] = 1
                U = P @ U @ P.T
                q0, q1 = q1, q0
            S = np.zeros((4, 4))
            for a in range(2):
                for b in range(2):
                    S[b * 2 + a, a * 2 + b] = 1
            for t in range(q1 - 1, q0, -1):
                self.apply_gate(t, S)
            self.apply_gate(q0, U)
            for t in range(q0 + 1, q1):
                self.apply_gate(t, S)
            return
        if len(qubits) == 2 and abs(qubits[1] - qubits[0]) == 2:
            q0, q1 = qubits
            if q0 > q1:  # reorder so the gate acts on increasing sites
                P = np.zeros((4, 4))
                for a in range(2):
                    for b in range(2):
                        P[b * 2 + a, a * 2 + b] = 1
                U = P @ U @ P.T
                q0, q1 = q1, q0
            U8 = np.zeros((8, 8), dtype=np.complex128)
            for i in range(2):
                for j in range(2):
                    for k in range(2):
                        for l in range(2):
                            for m in range(2):
                                U8[i * 4 + m * 2 + j, k * 4 + m * 2 + l] = U[i * 2 + j, k * 2 + l]
            self.apply_gate(q0, U8)
            return
        raise NotImplementedError("only adjacent gates and distance-2 two-qubit gates")

    def amplitude(self, bits) -> complex:
        b = bytes(bytearray(int(x) & 1 for x in bits))
        out = np.zeros(2)
        lib().oracle_mps_amplitude(self._h, b, _dp(out))
        return complex(out[0], out[1])

    def expectation(self, site: int, O) -> complex:
        O = _c128(O)
        k = {2: 1, 4: 2, 8: 3}[O.shape[0]]
        out = np.zeros(2)
        rc = lib().oracle_mps_expectation(self._h, site, k, _dp(O.view(np.float64)), _dp(out))
        if rc != 0:
            raise RuntimeError("oracle expectation failed")
        return complex(out[0], out[1])

    def reduced_density(self, qubits) -> np.ndarray:
        q = np.ascontiguousarray(np.asarray(qubits, dtype=np.int32))
        d = 1 << len(q)
        rho = np.zeros((d, d), dtype=np.complex128)
        rc = lib().oracle_mps_reduced_density(self._h, _ip(q), len(q), _dp(rho.view(np.float64)))
        if rc != 0:
            raise RuntimeError("oracle rdo failed")
        return rho

    def sample(self, u) -> np.ndarray:
        """Bit strings (rows) from uniforms u (rows of n values in [0, 1))."""
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, self.n))
        out = np.zeros(u.shape, dtype=np.uint8)
        buf = ctypes.create_string_buffer(self.n)
        for r in range(u.shape[0]):
            lib().oracle_mps_sample(self._h, _dp(u[r]), buf)
            out[r] = np.frombuffer(buf.raw[:self.n], dtype=np.uint8)
        return out

    def pauli_expectation(self, p: str) -> complex:
        assert len(p) == self.n and set(p) <= set("IXYZ")
        out = np.zeros(2)
        lib().oracle_mps_pauli(self._h, p.encode(), _dp(out))
        return complex(out[0], out[1])

    def bond_dim(self, b: int) -> int:
        return lib().oracle_mps_bond_dim(self._h, b)

    def schmidt(self, b: int) -> np.ndarray:
        out = np.zeros(self.bond_dim(b))
        lib().oracle_mps_get_schmidt(self._h, b, _dp(out))
        return out

    def last_diag(self):
        k = ctypes.c_int()
        w = ctypes.c_double()
        sw = ctypes.c_int()
        st = ctypes.c_int()
        lib().oracle_mps_last_diag(self._h, ctypes.byref(k), ctypes.byref(w), ctypes.byref(sw), ctypes.byref(st))
        return {"k": k.value, "discarded": w.value, "sweeps": sw.value, "status": st.value}

    def get_state(self):
        """(chi[n+1], [Gamma_s (2, chi_s, chi_{s+1})], [Lambda_b])."""
        chi = np.zeros(self.n + 1, dtype=np.int32)
        lib().oracle_mps_get_state(self._h, _ip(chi), None, None)
        ng = sum(2 * int(chi[s]) * int(chi[s + 1]) for s in range(self.n))
        nl = sum(int(chi[b + 1]) for b in range(self.n - 1))
        g = np.zeros(ng, dtype=np.complex128)
        lam = np.zeros(max(nl, 1))
        lib().oracle_mps_get_state(self._h, _ip(chi), _dp(g.view(np.float64)), _dp(lam))
        gammas, off = [], 0
        for s in range(self.n):
            sz = 2 * int(chi[s]) * int(chi[s + 1])
            gammas.append(g[off:off + sz].reshape(2, int(chi[s]), int(chi[s + 1])).copy())
            off += sz
        lams, off = [], 0
        for b in range(self.n - 1):
            lams.append(lam[off:off + int(chi[b + 1])].copy())
            off += int(chi[b + 1])
        return chi, gammas, lams

    def set_state(self, gammas, lams) -> None:
        chi = np.array([1] + [g.shape[2] for g in gammas], dtype=np.int32)
        g = _c128(np.concatenate([np.ravel(x) for x in gammas]))
        lam = np.ascontiguousarray(np.concatenate([np.ravel(x) for x in lams]) if lams else np.zeros(1))
        rc = lib().oracle_mps_set_state(self._h, _ip(chi), _dp(g.view(np.float64)), _dp(lam))
        if rc != 0:
            raise ValueError("bad state")
