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


def rng_for(config: int, circuit: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + 1000 * config + circuit)


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


# ---------------------------------------------------------------- configs ---

CONFIGS = {
    1: dict(name="n10_d10_u4_chi32", n=10, depth=10, chi_max=32, cutoff=1e-14),
    2: dict(name="n64_d20_u4_rz_chi256", n=64, depth=20, chi_max=256, cutoff=1e-12),
    3: dict(name="n48_d12_u8_ghz_chi128", n=48, depth=12, chi_max=128, cutoff=1e-12),
    4: dict(name="batch512_n16-64_d8-24_chi32-256", count=512, cutoff=1e-12),
    5: dict(name="n96_d30_u4_chi512_sketch", n=96, depth=30, chi_max=512, cutoff=1e-10),
}


def config_circuit(config: int, circuit: int = 0, n: int | None = None, depth: int | None = None):
    """Layers of the named workload (n, depth may be overridden for small cases)."""
    c = CONFIGS[config]
    rng = rng_for(config, circuit)
    n = c["n"] if n is None else n
    depth = c["depth"] if depth is None else depth
    if config == 1:
        return brickwork(n, depth, rng, first_u2_layer=True)
    if config == 2:
        return brickwork(n, depth, rng, rz_after_each=True)
    if config == 3:
        return ghz_prefix(n) + u8_shifted_brick(n, depth, rng)
    if config == 5:
        return brickwork(n, depth, rng)
    raise ValueError(config)


def batch_specs(count: int = 512, circuit_seed: int = 0):
    """Per-circuit (n, depth, chi_max) of the many-circuit workload."""
    rng = rng_for(4, circuit_seed)
    n = rng.integers(16, 65, size=count)
    d = rng.integers(8, 25, size=count)
    chi = rng.choice(np.array([32, 64, 128, 256]), size=count)
    return [(int(a), int(b), int(c)) for a, b, c in zip(n, d, chi)]


def batch_circuit(i: int, n: int, depth: int):
    return brickwork(n, depth, rng_for(4, 1 + i))


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
