"""Pins of the Hermitian-workload oracle (Sec. 2 diagonalisation; Sec. 2.1
exp_H, thermal state, pulse, <X> record, zero-padded |DFT|) against closed
forms: the 2 x 2 eigenproblem, the Heisenberg coupling's spectrum, the
exponential of a Pauli matrix, the Boltzmann weights of a diagonal H, the
analytic free-induction decay of the paper's two-spin example, and a pure
tone's DFT with Parseval's identity."""
import numpy as np
import pytest

from oracle import hermitian as O
from paper_1111_3124_gb300 import circuits as C


def test_heev_closed_forms():
    a, d, b = 1.3, -0.4, 0.7 - 0.2j
    w, V = O.heev([[a, b], [np.conj(b), d]])
    r = np.sqrt(((a - d) / 2) ** 2 + abs(b) ** 2)
    assert np.allclose(w, [(a + d) / 2 - r, (a + d) / 2 + r], atol=1e-15)
    heis = np.kron(C.X, C.X) + np.kron(C.Y, C.Y) + np.kron(C.Z, C.Z)
    w, V = O.heev(heis)
    assert np.allclose(w, [-3, 1, 1, 1], atol=1e-14)
    assert np.allclose(V @ np.diag(w) @ V.conj().T, heis, atol=1e-14)


def test_expm_of_a_pauli_matrix():
    th = 0.37
    E = O.expm(C.X, -1j * th)
    assert np.allclose(E, np.cos(th) * C.I2 - 1j * np.sin(th) * C.X, atol=1e-15)
    E = O.expm(C.Z, 0.8)
    assert np.allclose(E, np.diag([np.exp(0.8), np.exp(-0.8)]), atol=1e-14)


def test_thermal_state_of_a_diagonal_hamiltonian():
    ex = C.nmr_example()
    H, beta = ex["H"], ex["beta"]
    rho = O.thermal(H, beta)
    E = np.real(np.diag(H))
    p = np.exp(-beta * (E - E.min()))
    assert np.allclose(np.diag(rho).real, p / p.sum(), rtol=1e-13, atol=0)
    assert np.max(np.abs(rho - np.diag(np.diag(rho)))) == 0.0


def _fid_closed_form(ex, ms):
    """<X_1>(t) after the Y_90 pulse for H = w1 ZI + w2 IZ + J ZZ (Hz),
    evolution exp(-2 pi i H t): sum_b (rho_1b - rho_0b) cos(2 pi (2 w1 + 2 J z_b) t)."""
    rho = O.thermal(ex["H"], ex["beta"])
    d = np.real(np.diag(rho))  # index 2a + b
    t = np.asarray(ms) * ex["dt"]
    out = np.zeros(len(ms))
    for b, zb in ((0, 1.0), (1, -1.0)):
        out += (d[2 + b] - d[b]) * np.cos(2 * np.pi * (2 * ex["w1"] + 2 * ex["J"] * zb) * t)
    return out


def test_fid_of_the_two_spin_example_matches_the_closed_form():
    ex = C.nmr_example()
    assert ex["N"] == 32768
    rho = O.thermal(ex["H"], ex["beta"])
    ms = [0, 1, 17, 1000, 32767]
    s = O.fid(rho, 2 * np.pi * ex["H"], ex["O"], ex["dt"], ms, P=ex["P"])
    ref = _fid_closed_form(ex, ms)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(s.imag)) < 1e-12 * scale
    assert np.max(np.abs(s.real - ref)) < 1e-9 * scale


def test_dft_of_a_pure_tone_and_parseval():
    n_in, n_out, f0 = 256, 1024, 40
    x = np.exp(2j * np.pi * f0 * np.arange(n_in) / n_out)
    X = O.dft_abs(x, n_out)
    assert abs(X[f0] - n_in) < 1e-9
    assert np.argmax(X) == f0
    assert abs(np.sum(X ** 2) - n_out * np.sum(np.abs(x) ** 2)) < 1e-8 * n_out * n_in


def test_thermal_deviation_against_mpmath_at_300K():
    """rho - I/D at 300 K for Hz-scale couplings (beta ||H|| ~ 1e-10): the
    oracle's expm1 form against exp(-beta H) / Tr - I/D evaluated by mpmath at
    60 digits (where the cancellation against 1/D costs nothing)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    H = C.spin_hamiltonians(1, 3, np.random.default_rng(8))[0]
    beta = C.PLANCK / C.BOLTZMANN / 300.0
    dev = O.thermal_deviation(H, beta)
    M = mpmath.matrix([[mpmath.mpc(H[r, c].real, H[r, c].imag) for c in range(8)] for r in range(8)])
    E = mpmath.expm(-mpmath.mpf(beta) * M)
    tr = sum(E[i, i] for i in range(8))
    ref = np.array([[complex((E[r, c] / tr - (1 if r == c else 0) / mpmath.mpf(8))) for c in range(8)]
                    for r in range(8)])
    scale = np.max(np.abs(ref))
    assert scale < 1e-9  # the deviation is tiny against 1/D
    assert np.max(np.abs(dev - ref)) < 1e-13 * scale
    # the plain formula loses most digits of it
    plain = O.thermal(H, beta) - np.eye(8) / 8
    assert np.max(np.abs(plain - ref)) > 1e-9 * scale
