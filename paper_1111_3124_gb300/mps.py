"""Thin ctypes binding of the C ABI declared in include/mps.h.

Every step of the gate update runs in the CUDA library libmps_gb300.so; this
module only converts arguments. There is no CPU fallback: importing it
without the built library, or using it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmps_gb300.so")

MPS_OK = 0
MPS_ERR_ARG = -1
MPS_ERR_NOMEM = -2
MPS_ERR_CUDA = -3
MPS_ERR_NOCONVERGE = -4
MPS_ERR_TIMEOUT = -5
MPS_ERR_NOT_UNITARY = -6
MPS_ERR_TOO_LARGE = -7
PREC_FP64 = 0
PREC_SPLIT = 1
SVD_JACOBI = 0
SVD_SKETCH_MLP = 1
MLP_PARAMS = 1153

# every symbol include/mps.h declares
EXPORTS = [
    "mps_create", "mps_destroy", "mps_set_stream", "mps_set_mode", "mps_reset", "mps_apply_gate",
    "mps_apply_layer", "mps_apply_layer_device", "mps_profile", "mps_profile_read", "mps_amplitude", "mps_amplitudes", "mps_expectation", "mps_reduced_density",
    "mps_get_schmidt", "mps_bond_dims", "mps_export", "mps_import", "mps_diag", "mps_sync", "mps_last_error",
    "mps_gate2_update_noalloc", "mps_split_zgemm", "mps_apply_layer_multi",
    "mps_mlp_create", "mps_mlp_destroy", "mps_mlp_params", "mps_mlp_forward", "mps_mlp_loss_grad", "mps_mlp_train",
    "mps_layer_features", "mps_set_predictor", "mps_sketch_stats", "mps_set_limits", "mps_debug_fail_alloc",
    "mps_program_create", "mps_program_run", "mps_program_updates", "mps_program_destroy", "mps_set_tuning",
    "mps_sample", "mps_pauli_expectations", "mps_apply_gate_on",
    "mps_dd_create", "mps_dd_destroy", "mps_dd_reset", "mps_dd_set_stream", "mps_dd_set_limits",
    "mps_dd_apply_layer", "mps_dd_apply_layer_device", "mps_dd_sync", "mps_dd_bond_dims", "mps_dd_get_schmidt",
    "mps_dd_amplitudes", "mps_dd_stats",
    "mps_heev_batched", "mps_hermitian_function_batched", "mps_fid_batched", "mps_dft_abs_batched",
    "mps_hermitian_last_stats", "mps_debug_bounded_wait", "mps_debug_mark_timed_out",
]


class MPSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (status %d)" % (msg, code))
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libmps_gb300.so is not built: run __graft_entry__.build() "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    fp = ctypes.POINTER(ctypes.c_float)
    bp = ctypes.c_char_p
    sig = {
        "mps_create": [I, I, D, ctypes.POINTER(P)],
        "mps_destroy": [P],
        "mps_set_stream": [P, P],
        "mps_set_mode": [P, I, I, I],
        "mps_reset": [P],
        "mps_apply_gate": [P, I, I, dp],
        "mps_apply_layer": [P, I, I, ip, dp],
        "mps_apply_layer_device": [P, I, I, ip, P],
        "mps_profile": [P, I],
        "mps_profile_read": [P, I, dp, ctypes.POINTER(ctypes.c_longlong), dp, ctypes.POINTER(ctypes.c_longlong)],
        "mps_amplitude": [P, bp, dp],
        "mps_amplitudes": [P, I, bp, dp],
        "mps_expectation": [P, I, I, dp, dp],
        "mps_reduced_density": [P, ip, I, dp],
        "mps_get_schmidt": [P, I, dp, ip],
        "mps_bond_dims": [P, ip],
        "mps_export": [P, ip, dp, dp],
        "mps_import": [P, ip, dp, dp],
        "mps_diag": [P, I, ip, ip, dp, ip, ip],
        "mps_sync": [P],
        "mps_gate2_update_noalloc": [P, P, P, P, P, P, I, D, dp, P],
        "mps_split_zgemm": [I, I, I, P, ctypes.c_longlong, P, ctypes.c_longlong, P, ctypes.c_longlong, I, P],
        "mps_apply_layer_multi": [I, ctypes.POINTER(P), I, ip, ip, dp],
        "mps_mlp_create": [ctypes.c_ulonglong, ctypes.POINTER(P)],
        "mps_mlp_destroy": [P],
        "mps_mlp_params": [P, fp, fp],
        "mps_mlp_forward": [P, I, fp, fp],
        "mps_mlp_loss_grad": [P, I, fp, fp, fp, fp],
        "mps_mlp_train": [P, I, fp, fp, I, I, ctypes.c_float, ctypes.c_ulonglong, fp],
        "mps_layer_features": [P, I, I, ip, dp, fp],
        "mps_set_predictor": [P, P],
        "mps_sketch_stats": [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(ctypes.c_longlong)],
        "mps_set_limits": [P, I],
        "mps_set_tuning": [P, I, ip, ip, ip],
        "mps_sample": [P, I, dp, P],
        "mps_apply_gate_on": [P, I, ip, dp, I],
        "mps_pauli_expectations": [P, I, bp, dp],
        "mps_program_create": [I, ctypes.POINTER(P), I, ip, ip, ip, ip, P, ctypes.POINTER(P)],
        "mps_program_run": [P],
        "mps_program_updates": [P, ctypes.POINTER(ctypes.c_longlong)],
        "mps_program_destroy": [P],
        "mps_debug_fail_alloc": [ctypes.c_longlong],
        "mps_dd_create": [I, I, D, ctypes.POINTER(P)],
        "mps_dd_destroy": [P],
        "mps_dd_reset": [P],
        "mps_dd_set_stream": [P, P],
        "mps_dd_set_limits": [P, I],
        "mps_dd_apply_layer": [P, I, I, ip, dp, dp],
        "mps_dd_apply_layer_device": [P, I, I, ip, P, P, P],
        "mps_dd_sync": [P],
        "mps_dd_bond_dims": [P, ip],
        "mps_dd_get_schmidt": [P, I, dp, dp, ip],
        "mps_dd_amplitudes": [P, I, bp, dp],
        "mps_dd_stats": [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), dp],
        "mps_heev_batched": [I, I, P, P, P, P],
        "mps_hermitian_function_batched": [I, I, P, I, D, D, P, P],
        "mps_fid_batched": [I, I, P, P, P, P, D, I, P, P],
        "mps_dft_abs_batched": [I, I, P, I, P, P],
        "mps_hermitian_last_stats": [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)],
        "mps_debug_bounded_wait": [D, P],
        "mps_debug_mark_timed_out": [P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = I
    L.mps_last_error.restype = ctypes.c_char_p
    L.mps_last_error.argtypes = []
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _c128(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def check(rc: int):
    if rc != MPS_OK:
        raise MPSError(rc, load_library().mps_last_error().decode(errors="replace"))


class MPS:
    """An n-qubit MPS in Vidal form on the current CUDA device (|0...0> at creation)."""

    def __init__(self, n: int, chi_max: int, cutoff: float, prec: int = PREC_FP64, stream=None):
        L = load_library()
        h = ctypes.c_void_p()
        check(L.mps_create(n, chi_max, float(cutoff), ctypes.byref(h)))
        self._h = h
        self.n, self.chi_max, self.cutoff = n, chi_max, cutoff
        if prec != PREC_FP64:
            self.set_mode(prec)
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load_library().mps_destroy(h)
        self._h = None

    __del__ = close

    def set_stream(self, stream) -> None:
        """stream: a torch.cuda.Stream, an integer cudaStream_t, or None."""
        ptr = getattr(stream, "cuda_stream", stream)
        check(load_library().mps_set_stream(self._h, ctypes.c_void_p(ptr) if ptr else None))

    def set_mode(self, prec: int, slices: int = 0, svd_mode: int = 0) -> None:
        check(load_library().mps_set_mode(self._h, prec, slices, svd_mode))

    def reset(self) -> None:
        check(load_library().mps_reset(self._h))

    def set_limits(self, max_sweeps: int) -> None:
        check(load_library().mps_set_limits(self._h, max_sweeps))

    def set_tuning(self, table) -> None:
        """table: list of (nw_max, f32_block, mode), nw_max increasing; mode 0
        launches the fp32 sweeps per round, 1 per round with the rotation on
        the tensor cores, 2 all sweeps in one scheduled launch of 256-thread
        CTAs (the default), 3 the same with 384-thread CTAs."""
        nw = np.ascontiguousarray([t[0] for t in table] or [0], dtype=np.int32)
        bw = np.ascontiguousarray([t[1] for t in table] or [0], dtype=np.int32)
        tc = np.ascontiguousarray([t[2] for t in table] or [0], dtype=np.int32)
        check(load_library().mps_set_tuning(self._h, len(table), _ip(nw), _ip(bw), _ip(tc)))

    def apply_gate(self, site: int, U) -> None:
        U = _c128(U)
        k = {2: 1, 4: 2, 8: 3}[U.shape[0]]
        check(load_library().mps_apply_gate(self._h, site, k, _dp(U.view(np.float64))))

    def apply_layer(self, sites, Us) -> None:
        Us = _c128(Us)
        k = {2: 1, 4: 2, 8: 3}[Us.shape[-1]]
        s = np.ascontiguousarray(np.asarray(sites, dtype=np.int32))
        check(load_library().mps_apply_layer(self._h, k, len(s), _ip(s), _dp(Us.view(np.float64))))

    def apply_layer_device(self, sites, d_Us, k: int) -> None:
        """Gates already in device memory: d_Us is a CUDA tensor (complex128,
        shape (n_gates, 2^k, 2^k), contiguous) or an integer device address."""
        ptr = d_Us.data_ptr() if hasattr(d_Us, "data_ptr") else int(d_Us)
        s = np.ascontiguousarray(np.asarray(sites, dtype=np.int32))
        check(load_library().mps_apply_layer_device(self._h, k, len(s), _ip(s), ctypes.c_void_p(ptr)))

    def layer_features(self, sites, Us) -> np.ndarray:
        Us = _c128(Us)
        s = np.ascontiguousarray(np.asarray(sites, dtype=np.int32))
        X = np.zeros((len(s), 16), dtype=np.float32)
        check(load_library().mps_layer_features(self._h, 2, len(s), _ip(s), _dp(Us.view(np.float64)),
                                                X.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return X

    def set_predictor(self, predictor) -> None:
        check(load_library().mps_set_predictor(self._h, predictor._h if predictor is not None else None))
        self._predictor = predictor  # keep it alive

    def sketch_stats(self):
        a, b, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        check(load_library().mps_sketch_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"sketched": a.value, "accepted": b.value, "routed_full": c.value}

    def profile(self, enable: bool) -> None:
        check(load_library().mps_profile(self._h, 1 if enable else 0))

    def profile_read(self, kernel: int):
        ms, fl = ctypes.c_double(), ctypes.c_double()
        nl, na = ctypes.c_longlong(), ctypes.c_longlong()
        check(load_library().mps_profile_read(self._h, kernel, ctypes.byref(ms), ctypes.byref(nl),
                                              ctypes.byref(fl), ctypes.byref(na)))
        return {"ms": ms.value, "launches": nl.value, "flops": fl.value, "launches_all": na.value}

    def apply_gate_on(self, qubits, U, route: str = "embed") -> None:
        """Gate on listed qubits (first = most significant index bit), routed by
        the library (mps_apply_gate_on): neighbours directly; distance 2 as a
        U(8) with the identity on the middle qubit (route "embed") or by SWAP
        updates (route "swap"); farther by SWAP updates."""
        U = _c128(U)
        q = np.ascontiguousarray(np.asarray(qubits, dtype=np.int32))
        check(load_library().mps_apply_gate_on(self._h, len(q), _ip(q), _dp(U.view(np.float64)),
                                               0 if route == "embed" else 1))

    def amplitudes(self, bits) -> np.ndarray:
        b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8).reshape(-1, self.n))
        out = np.zeros((b.shape[0], 2))
        check(load_library().mps_amplitudes(self._h, b.shape[0], b.ctypes.data_as(ctypes.c_char_p), _dp(out)))
        return out[:, 0] + 1j * out[:, 1]

    def amplitude(self, bits) -> complex:
        return complex(self.amplitudes(np.asarray(bits).reshape(1, -1))[0])

    def expectation(self, site: int, O) -> complex:
        O = _c128(O)
        k = {2: 1, 4: 2, 8: 3}[O.shape[0]]
        out = np.zeros(2)
        check(load_library().mps_expectation(self._h, site, k, _dp(O.view(np.float64)), _dp(out)))
        return complex(out[0], out[1])

    def sample(self, u) -> np.ndarray:
        """Bit strings (rows, qubit 0 first) from uniforms u (rows of n values in [0, 1))."""
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, self.n))
        bits = np.zeros(u.shape, dtype=np.uint8)
        check(load_library().mps_sample(self._h, u.shape[0], _dp(u), ctypes.c_void_p(bits.ctypes.data)))
        return bits

    def pauli_expectations(self, strings) -> np.ndarray:
        """<P> for Pauli strings (each of length n over "IXYZ")."""
        strings = list(strings)
        assert all(len(p) == self.n for p in strings)
        buf = "".join(strings).encode()
        out = np.zeros((len(strings), 2))
        check(load_library().mps_pauli_expectations(self._h, len(strings), buf, _dp(out)))
        return out[:, 0] + 1j * out[:, 1]

    def reduced_density(self, qubits) -> np.ndarray:
        q = np.ascontiguousarray(np.asarray(qubits, dtype=np.int32))
        d = 1 << len(q)
        rho = np.zeros((d, d), dtype=np.complex128)
        check(load_library().mps_reduced_density(self._h, _ip(q), len(q), _dp(rho.view(np.float64))))
        return rho

    def reduced_density_block(self, first: int, last: int) -> np.ndarray:
        return self.reduced_density(list(range(first, last + 1)))

    def schmidt(self, bond: int) -> np.ndarray:
        out = np.zeros(self.chi_max)
        ln = ctypes.c_int()
        check(load_library().mps_get_schmidt(self._h, bond, _dp(out), ctypes.byref(ln)))
        return out[:ln.value].copy()

    def bond_dims(self) -> np.ndarray:
        c = np.zeros(max(self.n - 1, 1), dtype=np.int32)
        check(load_library().mps_bond_dims(self._h, _ip(c)))
        return c[:self.n - 1]

    def export(self):
        chi = np.zeros(self.n + 1, dtype=np.int32)
        L = load_library()
        check(L.mps_export(self._h, _ip(chi), None, None))
        ng = sum(2 * int(chi[s]) * int(chi[s + 1]) for s in range(self.n))
        nl = sum(int(chi[b + 1]) for b in range(self.n - 1))
        g = np.zeros(ng, dtype=np.complex128)
        lam = np.zeros(max(nl, 1))
        check(L.mps_export(self._h, _ip(chi), _dp(g.view(np.float64)), _dp(lam)))
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

    def import_state(self, gammas, lams) -> None:
        chi = np.ascontiguousarray(np.array([1] + [g.shape[2] for g in gammas], dtype=np.int32))
        g = _c128(np.concatenate([np.ravel(x) for x in gammas]))
        lam = np.ascontiguousarray(np.concatenate([np.ravel(x) for x in lams]) if lams else np.zeros(1))
        check(load_library().mps_import(self._h, _ip(chi), _dp(g.view(np.float64)), _dp(lam)))

    def diag(self):
        cnt = ctypes.c_int()
        L = load_library()
        check(L.mps_diag(self._h, 0, ctypes.byref(cnt), None, None, None, None))
        m = cnt.value
        k = np.zeros(max(m, 1), dtype=np.int32)
        w = np.zeros(max(m, 1))
        sw = np.zeros(max(m, 1), dtype=np.int32)
        ks = np.zeros(max(m, 1), dtype=np.int32)
        check(L.mps_diag(self._h, m, ctypes.byref(cnt), _ip(k), _dp(w), _ip(sw), _ip(ks)))
        return {"k": k[:m], "discarded": w[:m], "sweeps": sw[:m], "k_sketch": ks[:m]}

    def sync(self) -> None:
        check(load_library().mps_sync(self._h))

    def run_layers(self, layers) -> int:
        """Applies a circuit given as layers of (site, U); same-size gates of a
        layer go through one batched mps_apply_layer call. Returns the number of
        multi-qubit updates."""
        nup = 0
        for layer in layers:
            by_k = {}
            for site, U in layer:
                by_k.setdefault(U.shape[0], []).append((site, U))
            for d in sorted(by_k):
                gs = by_k[d]
                self.apply_layer([s for s, _ in gs], np.stack([_c128(U) for _, U in gs]))
                if d >= 4:
                    nup += len(gs)
        return nup


class Program:
    """A recorded circuit over one or more MPS, replayed as one CUDA graph
    (mps_program_create). passes: a list of (k, gates, d_Us), where gates is a
    list of (owner, site) (owner indexes `states`) and d_Us a CUDA complex128
    tensor of shape (len(gates), 2^k, 2^k)."""

    def __init__(self, states, passes):
        import torch
        self._states = list(states)
        ks = np.ascontiguousarray([k for k, _, _ in passes], dtype=np.int32)
        ng = np.ascontiguousarray([len(g) for _, g, _ in passes], dtype=np.int32)
        owners = np.ascontiguousarray([o for _, g, _ in passes for (o, _) in g] or [0], dtype=np.int32)
        sites = np.ascontiguousarray([s for _, g, _ in passes for (_, s) in g] or [0], dtype=np.int32)
        mats = [U.reshape(-1) for _, g, U in passes if len(g)]
        self._gates = torch.cat(mats) if mats else torch.zeros(1, dtype=torch.complex128, device="cuda")
        hs = (ctypes.c_void_p * len(states))(*[m._h.value for m in states])
        h = ctypes.c_void_p()
        check(load_library().mps_program_create(len(states), hs, len(passes), _ip(ks), _ip(ng), _ip(sites),
                                                _ip(owners), ctypes.c_void_p(self._gates.data_ptr()),
                                                ctypes.byref(h)))
        self._h = h

    def run(self) -> None:
        check(load_library().mps_program_run(self._h))

    @property
    def updates(self) -> int:
        u = ctypes.c_longlong()
        check(load_library().mps_program_updates(self._h, ctypes.byref(u)))
        return u.value

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load_library().mps_program_destroy(h)
        self._h = None

    __del__ = close


class MPSDD:
    """An n-qubit MPS in Vidal form held in double-word arithmetic (hi + lo,
    about 106 bits) on the current CUDA device, chi_max <= 32 (mps_dd_*).
    Gates are complex128 matrices (U_lo optional low parts)."""

    def __init__(self, n: int, chi_max: int, cutoff: float, stream=None):
        h = ctypes.c_void_p()
        check(load_library().mps_dd_create(n, chi_max, float(cutoff), ctypes.byref(h)))
        self._h = h
        self.n, self.chi_max, self.cutoff = n, chi_max, cutoff
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load_library().mps_dd_destroy(h)
        self._h = None

    __del__ = close

    def set_stream(self, stream) -> None:
        ptr = getattr(stream, "cuda_stream", stream)
        check(load_library().mps_dd_set_stream(self._h, ctypes.c_void_p(ptr) if ptr else None))

    def set_limits(self, max_sweeps: int) -> None:
        check(load_library().mps_dd_set_limits(self._h, max_sweeps))

    def reset(self) -> None:
        check(load_library().mps_dd_reset(self._h))

    def apply_layer(self, sites, Us, Us_lo=None) -> None:
        Us = _c128(Us)
        k = {2: 1, 4: 2}[Us.shape[-1]]
        s = np.ascontiguousarray(np.asarray(sites, dtype=np.int32))
        lo = None if Us_lo is None else _c128(Us_lo)
        check(load_library().mps_dd_apply_layer(self._h, k, len(s), _ip(s), _dp(Us.view(np.float64)),
                                                None if lo is None else _dp(lo.view(np.float64))))

    def apply_layer_device(self, sites, d_sites, d_Us, k: int, d_Us_lo=None) -> None:
        """d_sites: CUDA int32 tensor; d_Us (and d_Us_lo): CUDA complex128
        tensors of shape (n_gates, 2^k, 2^k); they must outlive the kernels."""
        s = np.ascontiguousarray(np.asarray(sites, dtype=np.int32))
        lo = ctypes.c_void_p(d_Us_lo.data_ptr()) if d_Us_lo is not None else None
        check(load_library().mps_dd_apply_layer_device(self._h, k, len(s), _ip(s), ctypes.c_void_p(d_sites.data_ptr()),
                                                       ctypes.c_void_p(d_Us.data_ptr()), lo))

    def run_layers(self, layers) -> int:
        """Layers of (site, U); within a layer the U(2) gates are applied
        before the U(4) gates (they act on disjoint qubits). Returns the
        number of two-site updates."""
        nup = 0
        for layer in layers:
            by_k = {}
            for site, U in layer:
                by_k.setdefault(U.shape[0], []).append((site, U))
            for d in sorted(by_k):
                gs = by_k[d]
                self.apply_layer([s for s, _ in gs], np.stack([_c128(U) for _, U in gs]))
                if d == 4:
                    nup += len(gs)
        return nup

    def sync(self) -> None:
        check(load_library().mps_dd_sync(self._h))

    def bond_dims(self) -> np.ndarray:
        chi = np.zeros(self.n + 1, dtype=np.int32)
        check(load_library().mps_dd_bond_dims(self._h, _ip(chi)))
        return chi

    def schmidt(self, bond: int):
        """(hi, lo) arrays of Lambda_bond."""
        hi = np.zeros(self.chi_max)
        lo = np.zeros(self.chi_max)
        k = ctypes.c_int()
        check(load_library().mps_dd_get_schmidt(self._h, bond, _dp(hi), _dp(lo), ctypes.byref(k)))
        return hi[:k.value].copy(), lo[:k.value].copy()

    def amplitudes(self, bits) -> np.ndarray:
        """(count, 4) array: re hi, re lo, im hi, im lo."""
        b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8).reshape(-1, self.n))
        out = np.zeros((b.shape[0], 4))
        check(load_library().mps_dd_amplitudes(self._h, b.shape[0], b.ctypes.data_as(ctypes.c_char_p), _dp(out)))
        return out

    def stats(self) -> dict:
        u, s = ctypes.c_longlong(), ctypes.c_longlong()
        f = ctypes.c_double()
        check(load_library().mps_dd_stats(self._h, ctypes.byref(u), ctypes.byref(s), ctypes.byref(f)))
        return {"updates": u.value, "sweeps": s.value, "flops": f.value}


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_ptr(stream):
    ptr = getattr(stream, "cuda_stream", stream)
    return ctypes.c_void_p(ptr) if ptr else None


def _herm_batch(H):
    import torch
    H = H.to(torch.complex128).contiguous()
    if H.dim() == 2:
        H = H.unsqueeze(0)
    assert H.is_cuda and H.shape[-1] == H.shape[-2]
    return H


def heev(H, stream=None):
    """Eigenvalues (ascending) and eigenvectors (columns) of Hermitian CUDA
    matrices H (..., D, D) by the batched two-sided Jacobi kernel."""
    import torch
    Hb = _herm_batch(H)
    b, D = Hb.shape[0], Hb.shape[-1]
    w = torch.empty((b, D), dtype=torch.float64, device=Hb.device)
    V = torch.empty((b, D, D), dtype=torch.complex128, device=Hb.device)
    check(load_library().mps_heev_batched(b, D, _dptr(Hb), _dptr(w), _dptr(V), _stream_ptr(stream)))
    return w, V


def expm_hermitian(H, a: complex, stream=None):
    """exp(a H) for Hermitian CUDA matrices H (..., D, D), complex scalar a."""
    import torch
    Hb = _herm_batch(H)
    out = torch.empty_like(Hb)
    a = complex(a)
    check(load_library().mps_hermitian_function_batched(Hb.shape[0], Hb.shape[-1], _dptr(Hb), 0, a.real, a.imag,
                                                        _dptr(out), _stream_ptr(stream)))
    return out


def thermal_state(H, beta: float, stream=None):
    """exp(-beta H) / Tr exp(-beta H) for Hermitian CUDA matrices H."""
    import torch
    Hb = _herm_batch(H)
    out = torch.empty_like(Hb)
    check(load_library().mps_hermitian_function_batched(Hb.shape[0], Hb.shape[-1], _dptr(Hb), 1, float(beta), 0.0,
                                                        _dptr(out), _stream_ptr(stream)))
    return out


def thermal_deviation(H, beta: float, stream=None):
    """exp(-beta H) / Tr exp(-beta H) - I/D, accurate when beta ||H|| is small."""
    import torch
    Hb = _herm_batch(H)
    out = torch.empty_like(Hb)
    check(load_library().mps_hermitian_function_batched(Hb.shape[0], Hb.shape[-1], _dptr(Hb), 2, float(beta), 0.0,
                                                        _dptr(out), _stream_ptr(stream)))
    return out


def fid(rho, H, O, dt: float, N: int, P=None, stream=None):
    """Tr(exp(-iHt) P rho P^H exp(iHt) O) at t = m dt, m < N: (batch, N) complex128."""
    import torch
    r, Hb, Ob = _herm_batch(rho), _herm_batch(H), _herm_batch(O)
    Pb = _herm_batch(P) if P is not None else None
    b, D = Hb.shape[0], Hb.shape[-1]
    sig = torch.empty((b, N), dtype=torch.complex128, device=Hb.device)
    check(load_library().mps_fid_batched(b, D, _dptr(r), _dptr(Hb), _dptr(Ob), _dptr(Pb), float(dt), int(N),
                                         _dptr(sig), _stream_ptr(stream)))
    return sig


def hermitian_last_stats() -> dict:
    """Largest sweep count and total rotations of the last diagonalisation."""
    sw, rot = ctypes.c_longlong(), ctypes.c_longlong()
    check(load_library().mps_hermitian_last_stats(ctypes.byref(sw), ctypes.byref(rot)))
    return {"max_sweeps": sw.value, "rotations": rot.value}


def dft_abs(x, n_out: int, stream=None):
    """|DFT| of complex CUDA records x (batch, n_in) zero-padded to n_out."""
    import torch
    xb = x.to(torch.complex128).contiguous()
    if xb.dim() == 1:
        xb = xb.unsqueeze(0)
    out = torch.empty((xb.shape[0], n_out), dtype=torch.float64, device=xb.device)
    check(load_library().mps_dft_abs_batched(xb.shape[0], xb.shape[1], _dptr(xb), int(n_out), _dptr(out),
                                             _stream_ptr(stream)))
    return out


def circuit_passes(layers, owner: int = 0, device="cuda"):
    """A circuit given as layers of (site, U) as program passes: one pass per
    layer and gate size, gates on the device."""
    import torch
    out = []
    for layer in layers:
        by_k = {}
        for site, U in layer:
            by_k.setdefault({2: 1, 4: 2, 8: 3}[U.shape[0]], []).append((site, U))
        for k in sorted(by_k):
            gs = by_k[k]
            U = torch.from_numpy(np.ascontiguousarray(np.stack([_c128(u) for _, u in gs]))).to(device)
            out.append((k, [(owner, s) for s, _ in gs], U))
    return out


def debug_bounded_wait(limit_ms: float, stream=None) -> None:
    """Test hook: a bounded device wait on a barrier nothing completes; raises
    MPSError(MPS_ERR_TIMEOUT) when the wait runs out, as intended."""
    check(load_library().mps_debug_bounded_wait(float(limit_ms), _stream_ptr(stream)))


def debug_mark_timed_out(m) -> None:
    """Test hook: marks an MPS as if its split GEMM had timed out."""
    check(load_library().mps_debug_mark_timed_out(m._h))


def debug_fail_alloc(after: int) -> None:
    """Test hook: the allocation after the next `after` ones fails (-1: off)."""
    check(load_library().mps_debug_fail_alloc(int(after)))


def gate2_update_noalloc(gamma_l, gamma_r, lambda_l, lambda_m, lambda_r, chi, chi_max: int, cutoff: float, U,
                         stream=None) -> None:
    """Two-site update on caller-owned CUDA tensors (torch tensors: complex128
    [2, chi_max, chi_max] Gammas, float64 [chi_max] Lambdas, int32 [3] chi),
    with no device allocation by the library (see include/mps.h)."""
    U = _c128(U)
    s = getattr(stream, "cuda_stream", stream)
    check(load_library().mps_gate2_update_noalloc(
        ctypes.c_void_p(gamma_l.data_ptr()), ctypes.c_void_p(gamma_r.data_ptr()),
        ctypes.c_void_p(lambda_l.data_ptr()), ctypes.c_void_p(lambda_m.data_ptr()),
        ctypes.c_void_p(lambda_r.data_ptr()), ctypes.c_void_p(chi.data_ptr()), chi_max, float(cutoff),
        _dp(U.view(np.float64)), ctypes.c_void_p(s) if s else None))


def split_zgemm(A, B, slices: int = 8, stream=None):
    """C = A @ B for CUDA complex128 torch tensors (2-D) by the split-precision
    tensor-core GEMM. Returns a new tensor."""
    import torch
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    At = A.t().contiguous()  # column-major A
    Bt = B.t().contiguous()
    Ct = torch.empty((N, M), dtype=torch.complex128, device=A.device)
    s = getattr(stream, "cuda_stream", stream)
    check(load_library().mps_split_zgemm(M, N, K, ctypes.c_void_p(At.data_ptr()), M, ctypes.c_void_p(Bt.data_ptr()),
                                         K, ctypes.c_void_p(Ct.data_ptr()), M, slices,
                                         ctypes.c_void_p(s) if s else None))
    return Ct.t()


def apply_layer_multi(states, layers_per_state) -> int:
    """One batched pass over the multi-qubit gates of several MPS.

    states: list of MPS (the first one's stream, workspace and mode are used);
    layers_per_state: for each MPS a list of (site, U) with U of one size k
    (2 or 3 qubits), disjoint within each MPS. Returns the number of gates."""
    ks = {U.shape[0] for layer in layers_per_state for (_, U) in layer}
    if not ks:
        return 0
    assert len(ks) == 1, "one gate size per call"
    k = {4: 2, 8: 3}[ks.pop()]
    hs = (ctypes.c_void_p * len(states))(*[m._h.value for m in states])
    n = np.ascontiguousarray([len(layer) for layer in layers_per_state], dtype=np.int32)
    sites = np.ascontiguousarray([s for layer in layers_per_state for (s, _) in layer], dtype=np.int32)
    Us = _c128(np.stack([U for layer in layers_per_state for (_, U) in layer]))
    check(load_library().mps_apply_layer_multi(len(states), hs, k, _ip(n), _ip(sites), _dp(Us.view(np.float64))))
    return int(n.sum())


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class RankPredictor:
    """The 16-64-1 tanh MLP (fp32) trained and run by the library's kernels."""

    def __init__(self, seed: int = 0):
        h = ctypes.c_void_p()
        check(load_library().mps_mlp_create(seed, ctypes.byref(h)))
        self._h = h

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load_library().mps_mlp_destroy(h)
        self._h = None

    __del__ = close

    @property
    def params(self) -> np.ndarray:
        p = np.zeros(MLP_PARAMS, dtype=np.float32)
        check(load_library().mps_mlp_params(self._h, _fp(p), None))
        return p

    @params.setter
    def params(self, p) -> None:
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        check(load_library().mps_mlp_params(self._h, None, _fp(p)))

    def forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32).reshape(-1, 16))
        Y = np.zeros(X.shape[0], dtype=np.float32)
        check(load_library().mps_mlp_forward(self._h, X.shape[0], _fp(X), _fp(Y)))
        return Y

    def loss_grad(self, X, T):
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32).reshape(-1, 16))
        T = np.ascontiguousarray(np.asarray(T, dtype=np.float32))
        loss = np.zeros(1, dtype=np.float32)
        g = np.zeros(MLP_PARAMS, dtype=np.float32)
        check(load_library().mps_mlp_loss_grad(self._h, X.shape[0], _fp(X), _fp(T), _fp(loss), _fp(g)))
        return float(loss[0]), g

    def train(self, X, T, epochs: int = 20, batch: int = 256, lr: float = 1e-3, seed: int = 0) -> float:
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32).reshape(-1, 16))
        T = np.ascontiguousarray(np.asarray(T, dtype=np.float32))
        loss = np.zeros(1, dtype=np.float32)
        check(load_library().mps_mlp_train(self._h, X.shape[0], _fp(X), _fp(T), epochs, batch, lr, seed, _fp(loss)))
        return float(loss[0])
