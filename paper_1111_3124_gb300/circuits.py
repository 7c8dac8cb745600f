"""Seeded synthetic inputs: gates, circuits and Vidal-form states.

This module produces inputs only; it holds none of the gate-update arithmetic
and is shared by the tests, the benchmark and the CPU oracle's tests alike.

A circuit is a list of layers; a layer is a list of ``(site, U)`` with ``U`` a
``2^k x 2^k`` complex128 unitary acting on sites ``site..site+k-1`` (the first
site is the most significant bit of U's index, as in the Sec. 3.2 example).
Gates inside one layer act on disjoint sites.

Workload recipes (the paper ships no dataset; its elementary gate set is
U(2), U(4), U(8), Sec. 1):
  * Haar-random U(d): complex Ginibre matrix, QR, columns multiplied by the
    phase of R's diagonal (Mezzadri, Notices AMS 54, 592, 2007);
  * brickwork: even layers act on (0,1),(2,3),..., odd layers on (1,2),(3,4),...;
  * shifted brick of U(8): layer l acts on triples starting at (l mod 3) + 3j;
  * RZ(phi) = diag(e^{-i phi/2}, e^{+i phi/2}), phi ~ U[0, 2 pi);
  * GHZ ladder: H on qubit 0, then CNOT(q -> q+1) for q = 0..n-2.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20111114

H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def rng_for(group: int, circuit: int = 0) -> np.random.Generator:
    """The generator of circuit `circuit` of a workload's seed group."""
    return np.random.default_rng(SEED_BASE + 1000 * group + circuit)


def haar_unitary(d: int, rng: np.random.Generator) -> np.ndarray:
    g = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0)
    q, r = np.linalg.qr(g)
    ph = np.diag(r) / np.abs(np.diag(r))
    return np.ascontiguousarray(q * ph[None, :])


def rz(phi: float) -> np.ndarray:
    return np.diag([np.exp(-0.5j * phi), np.exp(0.5j * phi)]).astype(np.complex128)


def brickwork_sites(n: int, layer: int):
    return list(range(layer % 2, n - 1, 2))


def shifted_brick_sites(n: int, layer: int):
    return list(range(layer % 3, n - 2, 3))


def brickwork(n: int, depth: int, rng, first_u2_layer: bool = False, rz_after_each: bool = False):
    layers = []
    if first_u2_layer:
        layers.append([(q, haar_unitary(2, rng)) for q in range(n)])
    for l in range(depth):
        layers.append([(s, haar_unitary(4, rng)) for s in brickwork_sites(n, l)])
        if rz_after_each:
            layers.append([(q, rz(rng.uniform(0.0, 2 * np.pi))) for q in range(n)])
    return layers


def weak_gate(rng: np.random.Generator, t_max: float = 0.3) -> np.ndarray:
    """A weakly entangling U(4): exp(-i t (XX + YY + ZZ)), t ~ U[0, t_max),
    dressed with Haar-random single-qubit gates on both sides."""
    h = np.kron(X, X) + np.kron(Y, Y) + np.kron(Z, Z)
    w, v = np.linalg.eigh(h)
    t = rng.uniform(0.0, t_max)
    core = (v * np.exp(-1j * t * w)[None, :]) @ v.conj().T
    a = np.kron(haar_unitary(2, rng), haar_unitary(2, rng))
    b = np.kron(haar_unitary(2, rng), haar_unitary(2, rng))
    return np.ascontiguousarray(a @ core @ b)


def weak_brickwork(n: int, depth: int, rng, t_max: float = 0.3):
    """Brickwork of weakly entangling gates (Trotter-step-like circuits)."""
    return [[(s, weak_gate(rng, t_max)) for s in brickwork_sites(n, l)] for l in range(depth)]


def echo_brickwork(n: int, depth: int, rng, t_max: float = 0.3):
    """Loschmidt echo: a weakly entangling brickwork followed by its exact
    inverse (the layers reversed, each gate replaced by U^dagger). In the
    second half each update lowers the entanglement of its bond, so the kept
    rank falls well below theta's dimensions."""
    fwd = weak_brickwork(n, depth, rng, t_max)
    back = [[(s, np.ascontiguousarray(U.conj().T)) for s, U in layer] for layer in reversed(fwd)]
    return fwd + back


def ghz_prefix(n: int):
    layers = [[(0, H.copy())]]
    for q in range(n - 1):
        layers.append([(q, CNOT.copy())])
    return layers


def u8_shifted_brick(n: int, depth: int, rng):
    return [[(s, haar_unitary(8, rng)) for s in shifted_brick_sites(n, l)] for l in range(depth)]


# -------------------------------------------------------------- workloads ---

# The named workloads (sizes in the names); seed_group selects their seeds.
WORKLOADS = {
    "n10_d10_u4_chi32": dict(name="n10_d10_u4_chi32", n=10, depth=10, chi_max=32, cutoff=1e-14, seed_group=1,
                             kind="brickwork after a layer of U(2)"),
    "n64_d20_u4_rz_chi256": dict(name="n64_d20_u4_rz_chi256", n=64, depth=20, chi_max=256, cutoff=1e-12,
                                 seed_group=2, kind="brickwork with RZ phases after each layer"),
    "n48_d12_u8_ghz_chi128": dict(name="n48_d12_u8_ghz_chi128", n=48, depth=12, chi_max=128, cutoff=1e-12,
                                  seed_group=3, kind="GHZ prefix, then a shifted brick of U(8)"),
    "batch512_n16-64_d8-24_chi32-256": dict(name="batch512_n16-64_d8-24_chi32-256", count=512, cutoff=1e-12,
                                            seed_group=4, kind="512 brickwork circuits of random sizes"),
    "n96_d30_u4_chi512_sketch": dict(name="n96_d30_u4_chi512_sketch", n=96, depth=30, chi_max=512, cutoff=1e-10,
                                     seed_group=5, kind="brickwork"),
}
N10 = "n10_d10_u4_chi32"
N64_CHI256 = "n64_d20_u4_rz_chi256"
N48_U8 = "n48_d12_u8_ghz_chi128"


def workload_circuit(name: str, circuit: int = 0, n: int | None = None, depth: int | None = None):
    """Layers of the named workload (n, depth may be overridden for small cases)."""
    c = WORKLOADS[name]
    rng = rng_for(c["seed_group"], circuit)
    n = c["n"] if n is None else n
    depth = c["depth"] if depth is None else depth
    if name == N10:
        return brickwork(n, depth, rng, first_u2_layer=True)
    if name == N64_CHI256:
        return brickwork(n, depth, rng, rz_after_each=True)
    if name == N48_U8:
        return ghz_prefix(n) + u8_shifted_brick(n, depth, rng)
    if name == "n96_d30_u4_chi512_sketch":
        return brickwork(n, depth, rng)
    raise ValueError(name)


def batch_specs(count: int = 512, circuit_seed: int = 0):
    """Per-circuit (n, depth, chi_max) of the many-circuit workload."""
    rng = rng_for(WORKLOADS["batch512_n16-64_d8-24_chi32-256"]["seed_group"], circuit_seed)
    n = rng.integers(16, 65, size=count)
    d = rng.integers(8, 25, size=count)
    chi = rng.choice(np.array([32, 64, 128, 256]), size=count)
    return [(int(a), int(b), int(c)) for a, b, c in zip(n, d, chi)]


def batch_circuit(i: int, n: int, depth: int):
    return brickwork(n, depth, rng_for(WORKLOADS["batch512_n16-64_d8-24_chi32-256"]["seed_group"], 1 + i))


def count_updates(layers) -> int:
    return sum(1 for layer in layers for (s, U) in layer if U.shape[0] >= 4)


# --------------------------------------------------------- synthetic states ---

def random_vidal_state(n: int, chi, rng, decay: float = 8.0):
    """A synthetic Vidal-form state with prescribed bond dimensions.

    chi: sequence of n+1 bond dimensions with chi[0] = chi[n] = 1. Gamma
    entries are complex Gaussians scaled by 1/sqrt(2 chi_left); each Lambda is
    a positive, descending, unit-norm vector lambda_c ~ exp(-c/ decay*chi) with a
    random jitter. The state is not canonical: it is an input with the shapes
    and value ranges of a saturated simulation, used to time and compare single
    updates."""
    chi = [int(c) for c in chi]
    gammas = []
    for s in range(n):
        a, b = chi[s], chi[s + 1]
        g = (rng.standard_normal((2, a, b)) + 1j * rng.standard_normal((2, a, b))) / np.sqrt(4.0 * a)
        gammas.append(g.astype(np.complex128))
    lams = []
    for b in range(n - 1):
        m = chi[b + 1]
        x = np.exp(-np.arange(m) * decay / max(m, 1)) * (1.0 + 0.1 * rng.random(m))
        x = np.sort(x)[::-1]
        lams.append(x / np.linalg.norm(x))
    return gammas, lams


# ---- inputs for the double-word (about 106-bit) path ------------------------
# A binary64 gate is unitary only to about 1e-16, and a state evolved by such
# gates is normalised only to that level; to compare results at the 1e-30
# level the gates themselves must be unitary to that level. dd_unitary
# re-orthonormalises a binary64 gate's columns by Gram-Schmidt in Python's
# decimal arithmetic (60 digits) and returns each entry as hi + lo, two
# doubles whose exact sum is the entry to about 2^-106.

def _dec_split(x):
    from decimal import Decimal
    hi = float(x)
    lo = float(x - Decimal(hi))
    return hi, lo


def dd_unitary(U: np.ndarray):
    """(U_hi, U_lo), complex128 arrays with U_hi + U_lo unitary to ~1e-32,
    close to U (a binary64 unitary)."""
    from decimal import Decimal, localcontext
    U = np.asarray(U, dtype=np.complex128)
    d = U.shape[0]
    with localcontext() as ctx:
        ctx.prec = 60
        cols = [[(Decimal(float(U[r, c].real)), Decimal(float(U[r, c].imag))) for r in range(d)] for c in range(d)]
        out = []
        for c in range(d):
            v = cols[c]
            for q in out:  # v <- v - q (q^H v)
                pr = sum(a[0] * b[0] + a[1] * b[1] for a, b in zip(q, v))
                pi = sum(a[0] * b[1] - a[1] * b[0] for a, b in zip(q, v))
                v = [(b[0] - (a[0] * pr - a[1] * pi), b[1] - (a[0] * pi + a[1] * pr)) for a, b in zip(q, v)]
            nrm = sum(x * x + y * y for x, y in v).sqrt()
            out.append([(x / nrm, y / nrm) for x, y in v])
        hi = np.zeros((d, d), dtype=np.complex128)
        lo = np.zeros((d, d), dtype=np.complex128)
        for c in range(d):
            for r in range(d):
                rh, rl = _dec_split(out[c][r][0])
                ih, il = _dec_split(out[c][r][1])
                hi[r, c] = complex(rh, ih)
                lo[r, c] = complex(rl, il)
    return hi, lo


def dd_brickwork(n: int, depth: int, rng, rz_after_each: bool = True):
    """Brickwork of Haar U(4) (with RZ phases after each layer), every gate
    given as (site, U_hi, U_lo) through dd_unitary."""
    layers = []
    for layer in brickwork(n, depth, rng, rz_after_each=rz_after_each):
        layers.append([(s,) + dd_unitary(U) for s, U in layer])
    return layers


def dd_ghz_prefix(n: int):
    """H on qubit 0 (entries 1/sqrt(2) as hi + lo), then CNOT(q -> q+1)."""
    from decimal import Decimal, localcontext
    with localcontext() as ctx:
        ctx.prec = 60
        h, l = _dec_split(Decimal(1) / Decimal(2).sqrt())
    Hh = np.array([[h, h], [h, -h]], dtype=np.complex128)
    Hl = np.array([[l, l], [l, -l]], dtype=np.complex128)
    zero4 = np.zeros((4, 4), dtype=np.complex128)
    return [[(0, Hh, Hl)]] + [[(q, CNOT.copy(), zero4)] for q in range(n - 1)]


# ---- inputs for the Hermitian-matrix workload (the NMR example of Sec. 2.1) --
# Hamiltonians are in Hz; a state evolves by exp(-2 pi i H t) and the thermal
# state is exp(-beta H) / Tr with beta = h / (k_B T) (energy h * frequency).
PLANCK = 6.62606896e-34    # J s, the value Sec. 2.1 prints
BOLTZMANN = 1.3806504e-23  # J / K, the value Sec. 2.1 prints
Y90 = np.array([[1, 1], [-1, 1]], dtype=np.complex128) / np.sqrt(2.0)  # the Y_90 pulse of Sec. 2.1


def kron_all(*ms):
    out = np.ones((1, 1), dtype=np.complex128)
    for m in ms:
        out = np.kron(out, m)
    return out


def nmr_example():
    """The two-spin system of Sec. 2.1: a proton (w1 = 400 MHz) and a 13C spin
    (w2 = 125 MHz) with J12 = 140 kHz at T = 300 K;
    H = w1 Z(x)I + w2 I(x)Z + J12 Z(x)Z, the Y_90 pulse on the proton, <X> of
    the proton recorded every dt = 0.145 / w1 for N samples, N the power of
    two at or above 1 / (dt J12)."""
    w1, w2, J, T = 400e6, 125e6, 140e3, 300.0
    H = w1 * np.kron(Z, I2) + w2 * np.kron(I2, Z) + J * np.kron(Z, Z)
    dt = 0.145 / w1
    N = 1
    while N < 1.0 / dt / J:
        N *= 2
    return {"H": H, "P": np.kron(Y90, I2), "O": np.kron(X, I2), "beta": PLANCK / BOLTZMANN / T, "dt": dt, "N": N,
            "w1": w1, "w2": w2, "J": J, "T": T}


def spin_hamiltonians(count: int, spins: int, rng, shift_hz: float = 500.0, j_hz: float = 50.0):
    """`count` strongly coupled spin systems in the rotating frame:
    H = sum_k o_k Z_k + sum_{k<l} J_kl (X_k X_l + Y_k Y_l + Z_k Z_l) with offsets
    o_k ~ U[-shift_hz, shift_hz] and couplings J_kl ~ U[-j_hz, j_hz] (Hz);
    returns (count, 2^spins, 2^spins) complex128."""
    D = 1 << spins
    out = np.zeros((count, D, D), dtype=np.complex128)

    def op(P, k):
        return kron_all(*[P if q == k else I2 for q in range(spins)])

    Zs = [op(Z, k) for k in range(spins)]
    pairs = [(k, l) for k in range(spins) for l in range(k + 1, spins)]
    XYZ = {(k, l): op(X, k) @ op(X, l) + op(Y, k) @ op(Y, l) + Zs[k] @ Zs[l] for k, l in pairs}
    for b in range(count):
        o = rng.uniform(-shift_hz, shift_hz, spins)
        H = sum(o[k] * Zs[k] for k in range(spins))
        for kl in pairs:
            H = H + rng.uniform(-j_hz, j_hz) * XYZ[kl]
        out[b] = H
    return out


def random_hermitian(count: int, D: int, rng):
    g = rng.standard_normal((count, D, D)) + 1j * rng.standard_normal((count, D, D))
    return np.ascontiguousarray((g + np.conj(np.swapaxes(g, 1, 2))) / 2)
