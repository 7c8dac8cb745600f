"""Pins for the CPU oracle (no GPU): the paper's worked example, brute force,
closed forms, a library SVD and the binary128 mode.

Each pin is chosen so that a plausible slip in the oracle (a dropped Lambda, a
transposed gate index, a wrong sign in the complex rotation, a mis-ordered
reshape, a wrong truncation rule) fails at least one test here.
"""
import os

import numpy as np
import pytest

import oracle
from oracle.statevector import StateVector
from paper_1111_3124_gb300 import circuits as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def run_both(n, layers, chi_max=1 << 20, cutoff=0.0, prec=oracle.FP64):
    mps = oracle.OracleMPS(n, chi_max, cutoff, prec)
    sv = StateVector(n)
    for layer in layers:
        for site, U in layer:
            k = {2: 1, 4: 2, 8: 3}[U.shape[0]]
            mps.apply_gate(site, U)
            sv.apply(list(range(site, site + k)), U)
    return mps, sv


def mps_vector(mps, n):
    out = np.zeros(1 << n, dtype=np.complex128)
    for x in range(1 << n):
        bits = [(x >> (n - 1 - q)) & 1 for q in range(n)]
        out[x] = mps.amplitude(bits)
    return out


# ---------------------------------------------------------- worked example ---

def test_worked_example_sec32():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "worked_example_rdo.txt")) if l.strip() and not l.startswith("#")]
    m = oracle.OracleMPS(3, 8, 1e-14)
    init = m.reduced_density([0, 1, 2])
    exp_init = np.zeros((8, 8))
    for lab, nq, x, y, v in rows:
        if lab == "initial":
            exp_init[int(x, 2), int(y, 2)] = float(v)
    np.testing.assert_allclose(init, exp_init, atol=5e-8)
    m.apply_gate(0, C.H)
    m.apply_gate_on([0, 2], C.CNOT)
    rho = m.reduced_density([0, 2])
    exp = np.zeros((4, 4))
    for lab, nq, x, y, v in rows:
        if lab == "final":
            exp[int(x, 2), int(y, 2)] = float(v)
    # printed to 8 digits
    np.testing.assert_allclose(rho, exp, atol=5e-8)
    # the control is the first argument: CNOT(2 -> 0) would leave |00><10| terms
    assert abs(rho[0, 2]) < 1e-15


# ------------------------------------------------------------- dense SVD ---

@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (3, 5), (16, 16), (33, 17), (8, 40)])
def test_svd_against_lapack_and_identities(m, n):
    rng = np.random.default_rng(m * 100 + n)
    T = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    sigma, X, Y, sw = oracle.svd(T)
    assert sw > 0
    ref = np.linalg.svd(T, compute_uv=False)
    np.testing.assert_allclose(np.sort(sigma)[::-1], ref, rtol=0, atol=1e-13 * ref[0])
    np.testing.assert_allclose(X @ np.diag(sigma) @ Y.conj().T, T, atol=1e-13 * ref[0])
    r = min(m, n)
    np.testing.assert_allclose(X.conj().T @ X, np.eye(r), atol=1e-13)
    np.testing.assert_allclose(Y.conj().T @ Y, np.eye(r), atol=1e-13)


def test_svd_graded_spectrum_relative_accuracy():
    """Jacobi's hallmark: tiny singular values of a graded matrix are found to
    high relative accuracy (Demmel & Veselic 1992), which the Gram route would lose."""
    rng = np.random.default_rng(7)
    n = 24
    q1, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    s_true = np.logspace(0, -12, n)
    T = (q1 * s_true[None, :])  # columns scaled: T = Q diag(s), singular values s exactly up to rounding
    sigma, X, Y, _ = oracle.svd(T)
    np.testing.assert_allclose(np.sort(sigma)[::-1], s_true, rtol=1e-12)


def test_svd_binary128_closer_than_fp64():
    rng = np.random.default_rng(3)
    T = rng.standard_normal((12, 9)) + 1j * rng.standard_normal((12, 9))
    s64, *_ = oracle.svd(T, oracle.FP64)
    s128, X, Y, _ = oracle.svd(T, oracle.BINARY128)
    np.testing.assert_allclose(np.sort(s64), np.sort(s128), rtol=1e-14)
    # binary128 reconstruction is exact to the binary64 rounding of the outputs
    np.testing.assert_allclose(X @ np.diag(s128) @ Y.conj().T, T, atol=1e-15)


def test_svd_rank_deficient_and_zero():
    T = np.zeros((6, 4), dtype=np.complex128)
    s, X, Y, _ = oracle.svd(T)
    assert np.all(s == 0)
    u = np.arange(6) + 1j
    v = np.arange(4) - 2j
    s, X, Y, _ = oracle.svd(np.outer(u, v))
    ss = np.sort(s)[::-1]
    assert abs(ss[0] - np.linalg.norm(u) * np.linalg.norm(v)) < 1e-12 * ss[0]
    assert np.all(ss[1:] < 1e-13 * ss[0])


# ----------------------------------------------- MPS vs brute-force vector ---

def random_layers(n, depth, rng, ks=(1, 2, 3)):
    layers = []
    for _ in range(depth):
        layer, s = [], int(rng.integers(0, 2))
        while s < n:
            k = int(rng.choice(ks))
            if s + k > n:
                k = 1
            layer.append((s, C.haar_unitary(1 << k, rng)))
            s += k + int(rng.integers(0, 2))
        layers.append(layer)
    return layers


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mps_matches_statevector_mixed_gates(seed):
    rng = np.random.default_rng(100 + seed)
    n = 7
    mps, sv = run_both(n, random_layers(n, 6, rng))
    np.testing.assert_allclose(mps_vector(mps, n), sv.vector(), atol=1e-13)


def test_n10_brickwork_all_amplitudes_no_truncation():
    c = C.WORKLOADS[C.N10]
    layers = C.workload_circuit(C.N10)
    mps = oracle.OracleMPS(c["n"], c["chi_max"], c["cutoff"])
    sv = StateVector(c["n"])
    for layer in layers:
        for site, U in layer:
            k = {2: 1, 4: 2, 8: 3}[U.shape[0]]
            mps.apply_gate(site, U)
            sv.apply(list(range(site, site + k)), U)
            if k >= 2:
                d = mps.last_diag()
                assert d["status"] == 0 and d["discarded"] < 1e-26
    assert C.count_updates(layers) == 45
    v = mps_vector(mps, c["n"])
    np.testing.assert_allclose(v, sv.vector(), atol=1e-13)
    assert abs(np.linalg.norm(v) - 1) < 1e-13


def test_schmidt_vectors_are_schmidt_coefficients_eq2():
    rng = np.random.default_rng(11)
    n = 8
    mps, sv = run_both(n, random_layers(n, 5, rng, ks=(2,)))
    for b in range(n - 1):
        lam = mps.schmidt(b)
        ref = sv.schmidt(b)
        ref = ref[ref > 1e-14]
        assert len(lam) >= len(ref)
        np.testing.assert_allclose(np.sort(lam)[::-1][:len(ref)], ref, atol=1e-13)
        assert abs(np.sum(lam ** 2) - 1) < 1e-13


def test_expectation_and_rdo_vs_statevector():
    rng = np.random.default_rng(5)
    n = 6
    mps, sv = run_both(n, random_layers(n, 5, rng))
    for site, k in [(0, 1), (2, 2), (3, 3), (5, 1)]:
        O = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
        O = O + O.conj().T
        ref = sv.expectation(list(range(site, site + k)), O)
        assert abs(mps.expectation(site, O) - ref) < 1e-12
    for qs in ([0], [4, 1], [0, 2, 5], [5, 3, 1, 0]):
        np.testing.assert_allclose(mps.reduced_density(qs), sv.reduced_density(qs), atol=1e-13)


def test_binary128_mode_matches_and_is_tighter():
    rng = np.random.default_rng(9)
    n = 6
    layers = random_layers(n, 5, rng)
    m64, sv = run_both(n, layers)
    m128, _ = run_both(n, layers, prec=oracle.BINARY128)
    v64, v128, vs = mps_vector(m64, n), mps_vector(m128, n), sv.vector()
    np.testing.assert_allclose(v64, v128, atol=1e-13)
    # the binary128 run is limited only by the binary64 state vector it is compared to
    assert np.max(np.abs(v128 - vs)) <= np.max(np.abs(v64 - vs)) + 1e-15


# -------------------------------------------------------------- closed forms ---

def test_product_state_rank_one():
    rng = np.random.default_rng(1)
    n = 6
    layers = [[(q, C.haar_unitary(2, rng)) for q in range(n)],
              [(s, np.kron(C.haar_unitary(2, rng), C.haar_unitary(2, rng))) for s in (0, 2, 4)],
              [(s, np.kron(C.haar_unitary(2, rng), C.haar_unitary(2, rng))) for s in (1, 3)]]
    mps, sv = run_both(n, layers, chi_max=64, cutoff=1e-14)
    for b in range(n - 1):
        assert mps.bond_dim(b) == 1
        np.testing.assert_allclose(mps.schmidt(b), [1.0], atol=1e-14)
    np.testing.assert_allclose(mps_vector(mps, n), sv.vector(), atol=1e-14)


def test_bell_and_ghz_spectra():
    n = 12
    mps = oracle.OracleMPS(n, 128, 1e-12)
    for layer in C.ghz_prefix(n):
        for site, U in layer:
            mps.apply_gate(site, U)
    r = 1 / np.sqrt(2)
    for b in range(n - 1):
        np.testing.assert_allclose(mps.schmidt(b), [r, r], atol=1e-15)
    assert abs(mps.amplitude([0] * n) - r) < 1e-15
    assert abs(mps.amplitude([1] * n) - r) < 1e-15
    assert abs(mps.amplitude([1] + [0] * (n - 1))) < 1e-15


def test_unitarity_of_generated_gates():
    rng = np.random.default_rng(2)
    for d in (2, 4, 8):
        for _ in range(5):
            U = C.haar_unitary(d, rng)
            assert np.max(np.abs(U.conj().T @ U - np.eye(d))) < 1e-14


# ----------------------------------------------------------------- truncation ---

def _schmidt_gate(a, b):
    """U(4) whose first column is a|00> + b|11>, completed to a unitary."""
    M = np.eye(4, dtype=np.complex128)
    M[:, 0] = [a, 0, 0, b]
    q, r = np.linalg.qr(M)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


def test_truncation_to_chi_max_closed_form():
    U = _schmidt_gate(0.8, 0.6)
    m = oracle.OracleMPS(2, 1, 0.0)
    m.apply_gate(0, U)
    d = m.last_diag()
    assert d["k"] == 1 and abs(d["discarded"] - 0.36) < 1e-15
    np.testing.assert_allclose(m.schmidt(0), [1.0], atol=1e-15)
    assert abs(abs(m.amplitude([0, 0])) - 1) < 1e-14
    assert abs(m.amplitude([1, 1])) < 1e-15


@pytest.mark.parametrize("eps,kept", [(1e-13, 1), (1e-11, 2)])
def test_truncation_cutoff_rule(eps, kept):
    U = _schmidt_gate(np.sqrt(1 - eps ** 2), eps)
    m = oracle.OracleMPS(2, 8, 1e-12)
    m.apply_gate(0, U)
    assert m.bond_dim(0) == kept
    assert abs(np.sum(m.schmidt(0) ** 2) - 1) < 1e-15


def test_degenerate_cut_keeps_valid_state():
    """Bell state cut to chi_max = 1: the two Schmidt values tie; any one branch
    is a valid truncation. Unique: k = 1, discarded = 1/2, lambda = [1]."""
    m = oracle.OracleMPS(2, 1, 0.0)
    m.apply_gate(0, np.kron(C.H, C.I2))
    m.apply_gate(0, C.CNOT)
    d = m.last_diag()
    assert d["k"] == 1 and abs(d["discarded"] - 0.5) < 1e-15
    a00, a11 = abs(m.amplitude([0, 0])), abs(m.amplitude([1, 1]))
    assert abs(max(a00, a11) - 1) < 1e-14 and min(a00, a11) < 1e-15


def test_single_truncation_fidelity_equals_kept_weight():
    """From a canonical state, one truncation at one bond loses exactly the
    discarded weight: |<psi|psi_trunc>|^2 = 1 - w (Schmidt decomposition, Eq. 2),
    and the kept Schmidt values are the exact top-k, renormalised."""
    rng = np.random.default_rng(21)
    n = 8
    layers = random_layers(n, 6, rng, ks=(2,))
    exact, sv = run_both(n, layers)
    b = 3
    full = exact.schmidt(b)
    chi_b = len(full)
    k_cap = max(1, chi_b - 3)
    U = C.haar_unitary(4, rng)
    # reference: exact state after the extra gate
    sv.apply([b, b + 1], U)
    ref_s = sv.schmidt(b)
    trunc = oracle.OracleMPS(n, k_cap, 0.0)
    trunc.set_state(*exact.get_state()[1:])
    trunc.apply_gate(b, U)
    d = trunc.last_diag()
    w = float(np.sum(ref_s[k_cap:] ** 2))
    assert abs(d["discarded"] - w) < 1e-13
    np.testing.assert_allclose(trunc.schmidt(b), ref_s[:k_cap] / np.linalg.norm(ref_s[:k_cap]), atol=1e-13)
    v = mps_vector(trunc, n)
    f = abs(np.vdot(sv.vector(), v)) ** 2
    assert abs(f - (1 - w)) < 1e-12


def _top_k_projection(psi, n, bond, k):
    """The normalised projection of psi onto its k leading Schmidt vectors at
    the cut (0..bond)|(bond+1..n-1), its Schmidt values and the discarded weight."""
    m = psi.reshape(1 << (bond + 1), -1)
    u, s, vh = np.linalg.svd(m, full_matrices=False)
    w = float(np.sum(s[k:] ** 2) / np.sum(s ** 2))
    proj = (u[:, :k] * s[:k]) @ vh[:k]
    return proj.reshape(-1) / np.linalg.norm(proj), s, w


@pytest.mark.parametrize("seed,chi_max", [(31, 5), (32, 6), (33, 3)])
def test_three_site_truncation_is_two_successive_schmidt_projections(seed, chi_max):
    """A U(8) gate (Sec. 1, Sec. 3.1) whose two splits both truncate. From a
    canonical state the result is psi_2 = P_2 P_1 U psi (renormalised after
    each projection), P_1 keeping the chi_max leading Schmidt vectors of U psi
    at the first cut and P_2 those of the renormalised P_1 U psi at the second
    cut (Eq. 2). Pins both kept spectra, the summed discarded weight and every
    amplitude: a second split built from unweighted or mis-ordered first-split
    vectors, a lost renormalisation or a transposed reshape fails here."""
    rng = np.random.default_rng(seed)
    n, b = 8, 2
    layers = C.brickwork(n, 8, rng)
    exact, sv = run_both(n, layers)
    U = C.haar_unitary(8, rng)
    sv.apply([b, b + 1, b + 2], U)
    psi = sv.vector()
    psi1, s1, w1 = _top_k_projection(psi, n, b, chi_max)
    psi2, s2, w2 = _top_k_projection(psi1, n, b + 1, chi_max)
    assert len(s1) > chi_max and np.sum(s2 > 1e-12) > chi_max  # both splits truncate
    trunc = oracle.OracleMPS(n, chi_max, 0.0)
    trunc.set_state(*exact.get_state()[1:])
    trunc.apply_gate(b, U)
    d = trunc.last_diag()
    assert (trunc.bond_dim(b), trunc.bond_dim(b + 1), d["k"]) == (chi_max, chi_max, chi_max)
    np.testing.assert_allclose(trunc.schmidt(b), s1[:chi_max] / np.linalg.norm(s1[:chi_max]), atol=1e-13)
    np.testing.assert_allclose(trunc.schmidt(b + 1), s2[:chi_max] / np.linalg.norm(s2[:chi_max]), atol=1e-13)
    assert abs(d["discarded"] - (w1 + w2)) < 1e-13
    v = mps_vector(trunc, n)
    np.testing.assert_allclose(v, psi2, atol=1e-13)
    assert abs(np.vdot(v, v).real - 1.0) < 1e-13
    # the first split alone: |<U psi|psi_1>|^2 = 1 - w_1
    assert abs(abs(np.vdot(psi, psi1)) ** 2 - (1 - w1)) < 1e-13


def test_numerically_zero_values_dropped_with_zero_cutoff():
    """Exact zeros of a rank-deficient theta (a product gate on a product
    state) are dropped even with cutoff 0: the bond stays rank one and the
    state is exact."""
    m = oracle.OracleMPS(4, 16, 0.0)
    U = np.kron(C.H, C.H)
    m.apply_gate(1, U)
    assert [m.bond_dim(b) for b in range(3)] == [1, 1, 1]
    sv = StateVector(4)
    sv.apply([1, 2], U)
    np.testing.assert_allclose(mps_vector(m, 4), sv.vector(), atol=1e-15)


def test_schmidt_weights_sum_to_one_after_every_gate():
    """Eq. (2): every Lambda_b is a unit vector after every update, truncating
    or not (the kept values are renormalised, Sec. 3.1)."""
    rng = np.random.default_rng(71)
    n = 9
    m = oracle.OracleMPS(n, 6, 1e-3)  # chi_max 6 and a coarse cutoff: every layer truncates
    for layer in random_layers(n, 8, rng):
        for site, U in layer:
            m.apply_gate(site, U)
            for b in range(n - 1):
                lam = m.schmidt(b)
                assert abs(np.sum(lam ** 2) - 1.0) < 1e-14
                assert np.all(lam > 0) and np.all(np.diff(lam) <= 0)


def test_reduced_density_is_a_density_matrix():
    """RDO (Sec. 3.2) of a truncated state: Hermitian, unit trace, positive
    semidefinite, for one to four qubits in any listed order."""
    rng = np.random.default_rng(72)
    n = 8
    m = oracle.OracleMPS(n, 8, 1e-6)
    for layer in random_layers(n, 6, rng):
        for site, U in layer:
            m.apply_gate(site, U)
    for qs in ([3], [6, 1], [0, 4, 7], [5, 2, 3, 0]):
        rho = m.reduced_density(qs)
        np.testing.assert_allclose(rho, rho.conj().T, atol=1e-14)
        assert abs(np.trace(rho) - 1.0) < 1e-13
        assert np.min(np.linalg.eigvalsh(rho)) > -1e-13


def test_ghz_expectations_closed_form():
    """GHZ_n = (|0..0> + |1..1>)/sqrt 2: <Z_q> = 0, <Z_q Z_q+1> = 1,
    <X X X> on three neighbours = 0 for n > 3 and 1 for n = 3, and the
    one-qubit RDO is I/2."""
    Z = np.diag([1.0, -1.0]).astype(np.complex128)
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    for n in (3, 7):
        m = oracle.OracleMPS(n, 4, 1e-12)
        for layer in C.ghz_prefix(n):
            for site, U in layer:
                m.apply_gate(site, U)
        for q in range(n):
            assert abs(m.expectation(q, Z)) < 1e-14
        for q in range(n - 1):
            assert abs(m.expectation(q, np.kron(Z, Z)) - 1.0) < 1e-14
        xxx = m.expectation(0, np.kron(np.kron(X, X), X))
        assert abs(xxx - (1.0 if n == 3 else 0.0)) < 1e-14
        np.testing.assert_allclose(m.reduced_density([n // 2]), np.eye(2) / 2, atol=1e-15)


def test_echo_brickwork_returns_to_the_initial_state():
    """The Loschmidt-echo input (weak brickwork, then the layers reversed with
    U -> U^dagger) is the identity on the state vector, and its forward half
    entangles (a sanity check of the workload generator, no method arithmetic)."""
    n = 8
    layers = C.echo_brickwork(n, 6, np.random.default_rng(73), t_max=0.4)
    sv = StateVector(n)
    for layer in layers[:6]:
        for site, U in layer:
            sv.apply([site, site + 1], U)
    assert abs(sv.vector()[0]) < 0.999
    for layer in layers[6:]:
        for site, U in layer:
            sv.apply([site, site + 1], U)
    v = sv.vector()
    assert abs(abs(v[0]) - 1.0) < 1e-13 and np.max(np.abs(v[1:])) < 1e-13


# ------------------------------------------------- sampling, Pauli strings ---

PAULI = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]], dtype=complex),
         "Y": np.array([[0, -1j], [1j, 0]]), "Z": np.diag([1.0, -1.0]).astype(complex)}


def _brute_sample(psi, n, u):
    """Sequential conditional sampling from the normalised |psi|^2 (the
    marginal of the prefix over all suffixes), qubit 0 first; 0 if u < p0."""
    w = np.abs(psi.reshape((2,) * n)) ** 2
    bits = []
    for s in range(n):
        sub = w[tuple(bits)]
        m = sub.reshape(2, -1).sum(axis=1)
        b = 0 if u[s] < m[0] / m.sum() else 1
        bits.append(b)
    return np.array(bits, dtype=np.uint8)


def _pauli_brute(psi, n, p):
    op = np.array([[1.0]])
    for ch in p:
        op = np.kron(op, PAULI[ch])
    return np.vdot(psi, op @ psi) / np.vdot(psi, psi)


@pytest.mark.parametrize("chi_max", [64, 5])
def test_sampling_is_sequential_conditional_sampling_of_the_stored_state(chi_max):
    """With uniforms u the oracle's sample equals sequential sampling from the
    brute-force distribution |<b|psi>|^2 / <psi|psi> of the stored MPS (exact,
    or truncated and so not canonical)."""
    rng = np.random.default_rng(500 + chi_max)
    n = 8
    m = oracle.OracleMPS(n, chi_max, 0.0)
    for layer in random_layers(n, 6, rng):
        for site, U in layer:
            m.apply_gate(site, U)
    psi = mps_vector(m, n)
    u = rng.random((300, n))
    got = m.sample(u)
    for r in range(len(u)):
        assert np.array_equal(got[r], _brute_sample(psi, n, u[r]))


def test_pauli_strings_vs_statevector_and_truncated_state():
    rng = np.random.default_rng(515)
    n = 7
    layers = random_layers(n, 5, rng)
    exact, sv = run_both(n, layers)
    trunc = oracle.OracleMPS(n, 3, 0.0)
    for layer in layers:
        for site, U in layer:
            trunc.apply_gate(site, U)
    v_t = mps_vector(trunc, n)
    for _ in range(25):
        p = "".join(rng.choice(list("IXYZ"), size=n))
        assert abs(exact.pauli_expectation(p) - _pauli_brute(sv.vector(), n, p)) < 1e-13
        assert abs(trunc.pauli_expectation(p) - _pauli_brute(v_t, n, p)) < 1e-13


def test_pauli_strings_ghz_closed_forms():
    n = 9
    m = oracle.OracleMPS(n, 4, 0.0)
    for layer in C.ghz_prefix(n):
        for site, U in layer:
            m.apply_gate(site, U)
    assert abs(m.pauli_expectation("X" * n) - 1) < 1e-14
    assert abs(m.pauli_expectation("YY" + "X" * (n - 2)) + 1) < 1e-14   # Y Y on |11> gives -1
    assert abs(m.pauli_expectation("ZIIIIIIIZ") - 1) < 1e-14
    assert abs(m.pauli_expectation("IIIIZIIII")) < 1e-14
    # every string draws the GHZ pair (0...0, 1...1): a single X anywhere gives 0
    assert abs(m.pauli_expectation("IIXIIIIII")) < 1e-14


@pytest.mark.parametrize("route", ["embed", "swap"])
def test_non_adjacent_gates_by_routing_vs_statevector(route):
    """Sec. 3.2 applies two-qubit gates to non-neighbours: the oracle's routes
    (U(8) embedding at distance 2, SWAP chains) reproduce the state vector for
    every order and distance of the two qubits."""
    rng = np.random.default_rng(4400)
    n = 8
    m, sv = run_both(n, random_layers(n, 3, rng, ks=(2,)))
    for (a, b) in [(0, 2), (5, 3), (1, 6), (7, 0), (4, 3), (2, 7)]:
        U = C.haar_unitary(4, rng)
        m.apply_gate_on([a, b], U, route=route)
        sv.apply([a, b], U)
    np.testing.assert_allclose(mps_vector(m, n), sv.vector(), atol=1e-13)
