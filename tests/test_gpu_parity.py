"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: amplitudes |d amp| <= 1e-10 (absolute); Schmidt spectra
max |d lambda| <= 1e-12 * lambda_0; reconstructed two/three-site tensors
(gauge invariant where the cut has a spectral gap) within 1e-11 of their
largest entry. Both sides run the same algorithm in binary64, so the
differences are rounding only.
"""
import numpy as np
import pytest

import oracle
from oracle.statevector import StateVector
from paper_1111_3124_gb300 import circuits as C
from tests.helpers import (all_bits, oracle_run, random_state, spectrum_err, three_site_tensor,
                           two_site_tensor)

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-10
SPEC_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1111_3124_gb300 import build as B
    B.build()


def gpu_mps(n, chi_max, cutoff, prec=0):
    from paper_1111_3124_gb300.mps import MPS
    return MPS(n, chi_max, cutoff, prec)


# ------------------------------------------------------- paper's example ---

def test_worked_example_sec32_on_gpu():
    m = gpu_mps(3, 8, 1e-14)
    init = m.reduced_density_block(0, 2)
    assert abs(init[0, 0] - 1.0) < 1e-15 and np.sum(np.abs(init)) - 1.0 < 1e-15
    m.apply_gate(0, C.H)
    m.apply_gate_on([0, 2], C.CNOT)
    rho = m.reduced_density([0, 2])
    exp = np.zeros((4, 4))
    exp[0, 0] = exp[0, 3] = exp[3, 0] = exp[3, 3] = 0.5
    np.testing.assert_allclose(rho, exp, atol=5e-8)
    assert abs(rho[0, 2]) < 1e-15


# ------------------------------------------- n = 10 brickwork, all amplitudes ---

def test_n10_brickwork_all_amplitudes_vs_oracle_and_statevector():
    c = C.WORKLOADS[C.N10]
    n = c["n"]
    layers = C.workload_circuit(C.N10)
    g = gpu_mps(n, c["chi_max"], c["cutoff"])
    assert g.run_layers(layers) == 45
    ref = oracle_run(n, layers, c["chi_max"], c["cutoff"])
    sv = StateVector(n)
    for layer in layers:
        for site, U in layer:
            sv.apply(list(range(site, site + {2: 1, 4: 2, 8: 3}[U.shape[0]])), U)
    a = g.amplitudes(all_bits(n))
    err_sv = np.max(np.abs(a - sv.vector()))
    err_or = np.max(np.abs(a - np.array([ref.amplitude(b) for b in all_bits(n)])))
    assert err_sv < AMP_TOL and err_or < AMP_TOL, (err_sv, err_or)
    for b in range(n - 1):
        assert spectrum_err(g.schmidt(b), ref.schmidt(b)) < SPEC_TOL
        assert abs(np.sum(g.schmidt(b) ** 2) - 1) < 1e-13


def test_layer_diagnostics_no_truncation_in_the_n10_brickwork():
    c = C.WORKLOADS[C.N10]
    g = gpu_mps(c["n"], c["chi_max"], c["cutoff"])
    layers = C.workload_circuit(C.N10)
    for layer in layers:
        g.run_layers([layer])
        if layer[0][1].shape[0] == 4:
            d = g.diag()
            assert np.all(d["discarded"] < 1e-26)
            assert np.all(d["sweeps"] >= 1)


# ------------------------------------------------------ mixed gate sizes ---

@pytest.mark.parametrize("seed", [0, 1])
def test_mixed_1_2_3_site_gates_vs_statevector(seed):
    from tests.test_oracle import random_layers
    rng = np.random.default_rng(300 + seed)
    n = 8
    layers = random_layers(n, 6, rng)
    g = gpu_mps(n, 64, 0.0)
    for layer in layers:
        for site, U in layer:
            g.apply_gate(site, U)
    sv = StateVector(n)
    for layer in layers:
        for site, U in layer:
            sv.apply(list(range(site, site + {2: 1, 4: 2, 8: 3}[U.shape[0]])), U)
    np.testing.assert_allclose(g.amplitudes(all_bits(n)), sv.vector(), atol=AMP_TOL)


def test_expectation_and_rdo_vs_oracle():
    from tests.test_oracle import random_layers
    rng = np.random.default_rng(77)
    n = 7
    layers = random_layers(n, 5, rng)
    g = gpu_mps(n, 64, 1e-14)
    g.run_layers(layers)
    ref = oracle_run(n, layers, 64, 1e-14)
    for site, k in [(0, 1), (2, 2), (4, 3), (6, 1)]:
        O = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
        O = O + O.conj().T
        assert abs(g.expectation(site, O) - ref.expectation(site, O)) < 1e-11
    for qs in ([3], [5, 1], [0, 2, 6], [6, 4, 1, 0]):
        np.testing.assert_allclose(g.reduced_density(qs), ref.reduced_density(qs), atol=1e-12)


# --------------------------------------------------------------- closed forms ---

def test_ghz_prefix_closed_form_at_n48():
    c = C.WORKLOADS[C.N48_U8]
    n = c["n"]
    g = gpu_mps(n, c["chi_max"], c["cutoff"])
    g.run_layers(C.ghz_prefix(n))
    r = 1 / np.sqrt(2)
    for b in range(n - 1):
        np.testing.assert_allclose(g.schmidt(b), [r, r], atol=1e-15)
    assert abs(g.amplitude([0] * n) - r) < 1e-14
    assert abs(g.amplitude([1] * n) - r) < 1e-14


def test_product_state_rank_one():
    rng = np.random.default_rng(4)
    n = 12
    g = gpu_mps(n, 32, 1e-14)
    for s in range(0, n - 1, 2):
        g.apply_gate(s, np.kron(C.haar_unitary(2, rng), C.haar_unitary(2, rng)))
    for s in range(1, n - 1, 2):
        g.apply_gate(s, np.kron(C.haar_unitary(2, rng), C.haar_unitary(2, rng)))
    assert np.all(g.bond_dims() == 1)


# -------------------------------------------------------------- truncation ---

def test_truncating_circuit_vs_oracle():
    n, chi_max, cutoff = 12, 8, 1e-12
    layers = C.brickwork(n, 8, np.random.default_rng(55))
    g = gpu_mps(n, chi_max, cutoff)
    g.run_layers(layers)
    ref = oracle_run(n, layers, chi_max, cutoff)
    for b in range(n - 1):
        assert spectrum_err(g.schmidt(b), ref.schmidt(b)) < SPEC_TOL
    bits = np.random.default_rng(1).integers(0, 2, size=(64, n)).astype(np.uint8)
    a = g.amplitudes(bits)
    r = np.array([ref.amplitude(b) for b in bits])
    assert np.max(np.abs(a - r)) < AMP_TOL


def test_chi_max_one_closed_form():
    a, b = 0.8, 0.6
    M = np.eye(4, dtype=np.complex128)
    M[:, 0] = [a, 0, 0, b]
    q, r = np.linalg.qr(M)
    U = q * (np.diag(r) / np.abs(np.diag(r)))[None, :]
    g = gpu_mps(2, 1, 0.0)
    g.apply_gate(0, U)
    d = g.diag()
    assert d["k"][0] == 1 and abs(d["discarded"][0] - 0.36) < 1e-15
    assert abs(abs(g.amplitude([0, 0])) - 1) < 1e-14


@pytest.mark.parametrize("prec", [0, 1])
def test_degenerate_cut_keeps_a_valid_state(prec):
    """The oracle's tie pin on the GPU, in both modes: a Bell state cut to
    chi_max = 1. Its two Schmidt values tie, so either branch is a valid
    truncation; what is unique is compared: one kept value, discarded weight
    1/2, Lambda = [1], and a state that is one of the two branches. A larger
    case ties in the middle of the spectrum: GHZ on 6 qubits cut to chi_max = 1
    after the entangling prefix."""
    g = gpu_mps(2, 1, 0.0, prec)
    g.apply_gate(0, np.kron(C.H, C.I2))
    g.apply_gate(0, C.CNOT)
    d = g.diag()
    assert d["k"][0] == 1 and abs(d["discarded"][0] - 0.5) < 1e-14
    np.testing.assert_allclose(g.schmidt(0), [1.0], atol=1e-14)
    a = np.abs(g.amplitudes(np.array([[0, 0], [0, 1], [1, 0], [1, 1]], dtype=np.uint8)))
    assert abs(max(a[0], a[3]) - 1) < 1e-14 and min(a[0], a[3]) < 1e-15 and max(a[1], a[2]) < 1e-15
    n = 6
    h = gpu_mps(n, 1, 0.0, prec)
    for layer in C.ghz_prefix(n):
        for site, U in layer:
            h.apply_gate(site, U)
    for b in range(n - 1):
        np.testing.assert_allclose(h.schmidt(b), [1.0], atol=1e-14)
    amps = np.abs(h.amplitudes(all_bits(n)))
    assert abs(np.max(amps) - 1) < 1e-13 and np.sum(amps > 1e-13) == 1
    assert amps[np.argmax(amps)] == max(amps[0], amps[-1])  # a GHZ branch: all zeros or all ones


# --------------------------------------------- single updates, teacher forced ---

def single_update(chi, chi_max, site, d, seed, cutoff=1e-12):
    n = len(chi) - 1
    state = random_state(n, chi, seed)
    U = C.haar_unitary(d, np.random.default_rng(seed + 1))
    ref = oracle.OracleMPS(n, chi_max, cutoff)
    ref.set_state(*state)
    ref.apply_gate(site, U)
    g = gpu_mps(n, chi_max, cutoff)
    g.import_state(*state)
    g.apply_gate(site, U)
    return ref, g


@pytest.mark.parametrize("chi,chi_max", [((1, 3, 5, 2, 1), 64), ((1, 37, 45, 29, 1), 64),
                                         ((1, 70, 97, 50, 1), 128), ((1, 40, 40, 40, 1), 48)])
def test_single_two_site_update_ragged(chi, chi_max):
    """Random non-canonical Vidal state imported into both sides (spans
    several tiles and ragged tails); one U(4) on the middle bond. The last
    case truncates to chi_max (theta 80 x 80 kept to 48)."""
    ref, g = single_update(chi, chi_max, 1, 4, sum(chi))
    _, rg, rl = ref.get_state()
    _, gg, gl = g.export()
    assert len(gl[1]) == len(rl[1])
    assert spectrum_err(gl[1], rl[1]) < SPEC_TOL
    tg, tr = two_site_tensor(gg, gl, 1), two_site_tensor(rg, rl, 1)
    assert np.max(np.abs(tg - tr)) < 1e-11 * np.max(np.abs(tr))


@pytest.mark.parametrize("chi,chi_max", [((1, 9, 13, 11, 7, 1), 128), ((1, 33, 40, 21, 17, 1), 128),
                                         ((1, 20, 20, 20, 20, 1), 24)])
def test_single_three_site_update_ragged(chi, chi_max):
    """U(8) on sites 1..3 of a 5-site random state; the last case truncates
    both splits to chi_max."""
    ref, g = single_update(chi, chi_max, 1, 8, 7 * sum(chi))
    _, rg, rl = ref.get_state()
    _, gg, gl = g.export()
    for b in (1, 2):
        assert len(gl[b]) == len(rl[b])
        assert spectrum_err(gl[b], rl[b]) < SPEC_TOL
    tg, tr = three_site_tensor(gg, gl, 1), three_site_tensor(rg, rl, 1)
    assert np.max(np.abs(tg - tr)) < 1e-11 * np.max(np.abs(tr))


# ------------------------------------------------------------- edge cases ---

def test_edge_cases_small_n_and_errors():
    from paper_1111_3124_gb300.mps import MPSError
    g = gpu_mps(1, 4, 0.0)
    g.apply_gate(0, C.H)
    assert abs(g.amplitude([1]) - 1 / np.sqrt(2)) < 1e-15
    g3 = gpu_mps(3, 8, 0.0)
    U8 = C.haar_unitary(8, np.random.default_rng(3))
    g3.apply_gate(0, U8)
    np.testing.assert_allclose(g3.amplitudes(all_bits(3)), U8[:, 0], atol=1e-13)
    with pytest.raises(MPSError):
        g3.apply_gate(2, np.eye(4))  # out of range
    with pytest.raises(MPSError):
        g3.apply_gate(0, 2 * np.eye(4))  # not unitary
    with pytest.raises(MPSError):
        g3.apply_layer([0, 1], np.stack([np.eye(4)] * 2))  # overlap
    np.testing.assert_allclose(g3.amplitudes(all_bits(3)), U8[:, 0], atol=1e-13)  # untouched
    g3.apply_layer([], np.zeros((0, 4, 4)))  # empty layer


def test_rank_deficient_theta_exact_zeros():
    """A product gate on a product state: theta has rank 1 and exact zero
    singular values, which are dropped even with cutoff 0."""
    g = gpu_mps(4, 16, 0.0)
    g.apply_gate(1, np.kron(C.H, C.H))
    assert list(g.bond_dims()) == [1, 1, 1]


# -------------------------------------------- full-size single updates ---

def test_single_update_chi256_saturated():
    """One steady-state update of the n=64, chi_max=256 workload: theta
    512 x 512 truncated to 256, on a synthetic saturated state."""
    chi = (1, 256, 256, 256, 1)
    ref, g = single_update(chi, 256, 1, 4, 2024)
    _, rg, rl = ref.get_state()
    _, gg, gl = g.export()
    assert len(gl[1]) == len(rl[1]) == 256
    assert spectrum_err(gl[1], rl[1]) < SPEC_TOL
    tg, tr = two_site_tensor(gg, gl, 1), two_site_tensor(rg, rl, 1)
    assert np.max(np.abs(tg - tr)) < 1e-11 * np.max(np.abs(tr))


def test_single_three_site_update_chi128_saturated():
    chi = (1, 128, 128, 128, 128, 1)
    ref, g = single_update(chi, 128, 1, 8, 3031)
    _, rg, rl = ref.get_state()
    _, gg, gl = g.export()
    for b in (1, 2):
        assert spectrum_err(gl[b], rl[b]) < SPEC_TOL
    tg, tr = three_site_tensor(gg, gl, 1), three_site_tensor(rg, rl, 1)
    assert np.max(np.abs(tg - tr)) < 1e-11 * np.max(np.abs(tr))


@pytest.mark.parametrize("route", ["embed", "swap"])
def test_non_adjacent_gates_vs_statevector_and_oracle(route):
    """mps_apply_gate_on: every order and distance of the two qubits, exact
    (vs the state vector) and truncating (vs the oracle's same routing)."""
    rng = np.random.default_rng(4500)
    pairs = [(0, 2), (5, 3), (1, 6), (7, 0), (4, 3), (2, 7), (3, 5)]
    n = 8
    g = gpu_mps(n, 16, 0.0)
    sv = StateVector(n)
    for (a, b) in pairs:
        U = C.haar_unitary(4, rng)
        g.apply_gate_on([a, b], U, route=route)
        sv.apply([a, b], U)
    np.testing.assert_allclose(g.amplitudes(all_bits(n)), sv.vector(), atol=AMP_TOL)
    # truncating: n = 12, chi_max = 6
    n = 12
    g = gpu_mps(n, 6, 1e-12)
    o = oracle.OracleMPS(n, 6, 1e-12)
    for layer in C.brickwork(n, 3, rng):
        for site, U in layer:
            g.apply_gate(site, U)
            o.apply_gate(site, U)
    for (a, b) in [(0, 4), (9, 2), (5, 7), (11, 6)]:
        U = C.haar_unitary(4, rng)
        g.apply_gate_on([a, b], U, route=route)
        o.apply_gate_on([a, b], U, route=route)
    bits = np.random.default_rng(1).integers(0, 2, size=(64, n)).astype(np.uint8)
    np.testing.assert_allclose(g.amplitudes(bits), [o.amplitude(b) for b in bits], atol=AMP_TOL)
    for b in range(n - 1):
        assert spectrum_err(g.schmidt(b), o.schmidt(b)) < SPEC_TOL
