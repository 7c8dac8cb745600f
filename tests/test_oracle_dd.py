"""Pins of the oracle's binary128 mode at the 1e-30 level, the reference of
the double-word GPU path (the paper's multiprecision theme, Sec. 1 and the
256-bit setting of Sec. 3.2).

The oracle in binary128 is checked against a brute-force state vector and
SVDs computed by mpmath at 50 significant digits, on circuits whose gates are
unitary to ~1e-32 (circuits.dd_unitary: each entry given as hi + lo):
  * exact circuits: all amplitudes and every bond's spectrum (Eq. 2);
  * one truncating update from an exact state: the kept spectrum is the
    renormalised top-k of the exact Schmidt values, and every amplitude is
    the renormalised Schmidt projection of the exact state;
  * GHZ: every Schmidt value 1/sqrt(2) (closed form).
A mistake in the oracle that only shows beyond binary64 (a binary64
intermediate, an epsilon of the wrong format) fails these."""
import numpy as np
import pytest

import oracle
from paper_1111_3124_gb300 import circuits as C

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp


def _mpc(hi, lo=0j):
    return mpmath.mpc(hi.real, hi.imag) + mpmath.mpc(lo.real, lo.imag)


def _sv_apply(psi, n, site, k, Uh, Ul):
    """psi: list of 2^n mpc (qubit 0 the most significant bit)."""
    d = 1 << k
    U = [[_mpc(Uh[r, c], Ul[r, c]) for c in range(d)] for r in range(d)]
    out = list(psi)
    shift = n - site - k
    for x in range(1 << n):
        if (x >> shift) & (d - 1):
            continue
        idx = [x | (j << shift) for j in range(d)]
        v = [psi[i] for i in idx]
        for r in range(d):
            out[idx[r]] = mpmath.fsum(U[r][c] * v[c] for c in range(d))
    return out


def _schmidt(psi, n, b):
    rows, cols = 1 << (b + 1), 1 << (n - b - 1)
    M = mpmath.matrix(rows, cols)
    for x in range(1 << n):
        M[x // cols, x % cols] = psi[x]
    return sorted(mpmath.svd_c(M, compute_uv=False), reverse=True), M


def _hl(hi, lo):
    return [mpmath.mpf(h) + mpmath.mpf(l) for h, l in zip(hi, lo)]


def _amp_hl(o):
    return mpmath.mpc(mpmath.mpf(o[0]) + mpmath.mpf(o[1]), mpmath.mpf(o[2]) + mpmath.mpf(o[3]))


def _bits(x, n):
    return [(x >> (n - 1 - q)) & 1 for q in range(n)]


def test_dd_unitary_is_unitary_to_1e32():
    mp.dps = 50
    rng = np.random.default_rng(11)
    for d in (2, 4):
        U = C.haar_unitary(d, rng)
        hi, lo = C.dd_unitary(U)
        assert np.max(np.abs(hi - U)) < 1e-14
        M = mpmath.matrix([[_mpc(hi[r, c], lo[r, c]) for c in range(d)] for r in range(d)])
        E = M.H * M - mpmath.eye(d)
        assert max(abs(E[i, j]) for i in range(d) for j in range(d)) < 1e-31


def test_binary128_exact_circuit_against_mpmath_state_vector():
    mp.dps = 50
    n = 6
    layers = C.dd_brickwork(n, 6, np.random.default_rng(4242))
    m = oracle.OracleMPS(n, 64, 1e-30, oracle.BINARY128)
    psi = [mpmath.mpc(0)] * (1 << n)
    psi[0] = mpmath.mpc(1)
    for layer in layers:
        for site, Uh, Ul in layer:
            k = {2: 1, 4: 2}[Uh.shape[0]]
            m.apply_gate_hl(site, Uh, Ul)
            psi = _sv_apply(psi, n, site, k, Uh, Ul)
    amax = max(abs(a) for a in psi)
    err = max(abs(_amp_hl(m.amplitude_hl(_bits(x, n))) - psi[x]) for x in range(1 << n))
    assert err / amax < 1e-30, err
    for b in range(n - 1):
        ref, _ = _schmidt(psi, n, b)
        hi, lo = m.schmidt_hl(b)
        got = _hl(hi, lo)
        ref = [s for s in ref if s > mpmath.mpf(10) ** -25]
        assert len(got) == len(ref)
        assert max(abs(g - r) for g, r in zip(got, ref)) < 1e-30


def test_binary128_truncating_update_is_the_schmidt_projection():
    """Layer 1 entangles (0,1), (2,3), (4,5); a gate on (1,2) then needs
    bond 1 at rank 4 and chi_max = 2 keeps two values."""
    mp.dps = 50
    n, chi = 6, 2
    rng = np.random.default_rng(777)
    gates = [(s,) + C.dd_unitary(C.haar_unitary(4, rng)) for s in (0, 2, 4)]
    last = (1,) + C.dd_unitary(C.haar_unitary(4, rng))
    m = oracle.OracleMPS(n, chi, 1e-30, oracle.BINARY128)
    psi = [mpmath.mpc(0)] * (1 << n)
    psi[0] = mpmath.mpc(1)
    for site, Uh, Ul in gates + [last]:
        m.apply_gate_hl(site, Uh, Ul)
        psi = _sv_apply(psi, n, site, 2, Uh, Ul)
    sv, M = _schmidt(psi, n, 1)
    assert sv[3] > 1e-3  # rank 4 before truncation
    kept = sv[:chi]
    nk = mpmath.sqrt(mpmath.fsum(s * s for s in kept))
    hi, lo = m.schmidt_hl(1)
    got = _hl(hi, lo)
    assert max(abs(g - s / nk) for g, s in zip(got, kept)) < 1e-30
    # the truncated state: X_k Sigma_k Y_k^H / ||Sigma_k||
    U, S, V = mpmath.svd_c(M)
    rows, cols = M.rows, M.cols
    for x in range(1 << n):
        r, c = x // cols, x % cols
        ref = mpmath.fsum(U[r, j] * S[j] * V[j, c] for j in range(chi)) / nk
        assert abs(_amp_hl(m.amplitude_hl(_bits(x, n))) - ref) < 1e-30


def test_binary128_ghz_spectrum_is_one_over_sqrt2():
    mp.dps = 50
    n = 8
    m = oracle.OracleMPS(n, 4, 1e-30, oracle.BINARY128)
    for layer in C.dd_ghz_prefix(n):
        for site, Uh, Ul in layer:
            m.apply_gate_hl(site, Uh, Ul)
    r = 1 / mpmath.sqrt(2)
    for b in range(n - 1):
        hi, lo = m.schmidt_hl(b)
        got = _hl(hi, lo)
        assert len(got) == 2 and max(abs(g - r) for g in got) < 1e-32
    a = _amp_hl(m.amplitude_hl([1] * n))
    assert abs(a - r) < 1e-32
