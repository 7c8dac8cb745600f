"""Readout at scale on the GPU (Sec. 3.2's RDO and amplitudes): reduced
density operators of up to 12 qubits against the brute-force state vector and
the oracle, contracted from either end of the chain."""
import numpy as np
import pytest

import oracle
from oracle.statevector import StateVector
from paper_1111_3124_gb300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1111_3124_gb300 import build as B
    B.build()


def _exact_pair(n, depth, seed):
    from paper_1111_3124_gb300.mps import MPS
    rng = np.random.default_rng(seed)
    layers = C.brickwork(n, depth, rng)
    m = MPS(n, 1 << (n // 2), 0.0)
    m.run_layers(layers)
    sv = StateVector(n)
    for layer in layers:
        for site, U in layer:
            k = {2: 1, 4: 2, 8: 3}[U.shape[0]]
            sv.apply(list(range(site, site + k)), U)
    return m, sv


@pytest.mark.parametrize("qubits", [
    list(range(12)),                       # the whole chain: |psi><psi|
    [11, 10, 9, 8, 7, 6, 5, 4, 3, 2],      # ten qubits, reversed order
    [0, 5, 1, 9, 3, 11, 7],                # scattered, scrambled
    [0, 1, 2],                             # left end: contracted from the right
    [9, 10, 11],                           # right end: contracted from the left
])
def test_reduced_density_up_to_12_qubits_vs_statevector(qubits):
    m, sv = _exact_pair(12, 8, 404)
    rho = m.reduced_density(qubits)
    ref = sv.reduced_density(qubits)
    assert np.max(np.abs(rho - ref)) < 1e-13
    assert abs(np.trace(rho) - 1.0) < 1e-13


def test_reduced_density_of_a_truncated_state_vs_oracle():
    from paper_1111_3124_gb300.mps import MPS
    rng = np.random.default_rng(405)
    n = 14
    layers = C.brickwork(n, 10, rng)
    m = MPS(n, 12, 1e-12)
    m.run_layers(layers)
    orc = oracle.OracleMPS(n, 12, 1e-12)
    for layer in layers:
        for site, U in layer:
            orc.apply_gate(site, U)
    for q in ([2, 9, 4, 13], [6, 7, 8, 9, 10], [0, 13]):
        assert np.max(np.abs(m.reduced_density(q) - orc.reduced_density(q))) < 1e-11


def test_reduced_density_size_limits():
    from paper_1111_3124_gb300.mps import MPS, MPSError, MPS_ERR_TOO_LARGE
    m = MPS(16, 4, 0.0)
    with pytest.raises(MPSError) as e:
        m.reduced_density(list(range(13)))
    assert e.value.code == MPS_ERR_TOO_LARGE
    # 12 qubits of a product state: 4^12 blocks of 1 x 1 environments fit
    rho = m.reduced_density(list(range(2, 14)))
    assert abs(rho[0, 0] - 1.0) < 1e-15 and abs(np.sum(np.abs(rho)) - 1.0) < 1e-15


def _truncated_pair(n, chi_max, depth, seed, prec=0):
    from paper_1111_3124_gb300.mps import MPS
    rng = np.random.default_rng(seed)
    layers = C.brickwork(n, depth, rng, rz_after_each=True)
    m = MPS(n, chi_max, 1e-12, prec)
    m.run_layers(layers)
    orc = oracle.OracleMPS(n, chi_max, 1e-12)
    for layer in layers:
        for site, U in layer:
            orc.apply_gate(site, U)
    return m, orc, rng


@pytest.mark.parametrize("n,chi_max,prec", [(10, 32, 0), (20, 12, 0), (20, 12, 1)])
def test_sampling_matches_the_oracle_string_by_string(n, chi_max, prec):
    """Sequential conditional sampling with the same uniforms: every string
    equals the oracle's (exact state for n = 10, truncated for n = 20)."""
    m, orc, rng = _truncated_pair(n, chi_max, 8, 1700 + n, prec)
    u = rng.random((3000, n))
    got = m.sample(u)
    ref = orc.sample(u[:400])
    assert np.array_equal(got[:400], ref)
    # the empirical distribution of the rest follows |amp|^2 on the strings seen
    strings, counts = np.unique(got, axis=0, return_counts=True)
    top = np.argsort(-counts)[:5]
    amps = m.amplitudes(strings[top])
    p = np.abs(amps) ** 2
    emp = counts[top] / len(got)
    assert np.all(np.abs(emp - p) < 5 * np.sqrt(p * (1 - p) / len(got)) + 1e-3)


def test_sampling_a_ghz_state_gives_only_the_two_strings():
    from paper_1111_3124_gb300.mps import MPS
    n = 30
    m = MPS(n, 4, 0.0)
    m.run_layers(C.ghz_prefix(n))
    u = np.random.default_rng(3).random((2000, n))
    b = m.sample(u)
    assert np.all((b.sum(axis=1) == 0) | (b.sum(axis=1) == n))
    assert np.array_equal(b[:, 0] == 1, u[:, 0] >= 0.5)  # the first qubit decides, p = 1/2


def test_pauli_strings_vs_oracle_and_closed_forms():
    from paper_1111_3124_gb300.mps import MPS
    m, orc, rng = _truncated_pair(16, 10, 8, 1800)
    strings = ["".join(rng.choice(list("IXYZ"), size=16)) for _ in range(12)] + ["Z" * 16, "I" * 16]
    got = m.pauli_expectations(strings)
    for p, v in zip(strings, got):
        assert abs(v - orc.pauli_expectation(p)) < 1e-12
    n = 20
    g = MPS(n, 4, 0.0)
    g.run_layers(C.ghz_prefix(n))
    v = g.pauli_expectations(["X" * n, "YY" + "X" * (n - 2), "Z" + "I" * (n - 2) + "Z", "I" * 5 + "Z" + "I" * 14])
    np.testing.assert_allclose(v, [1, -1, 1, 0], atol=1e-13)


def test_sampling_and_pauli_reject_bad_input():
    from paper_1111_3124_gb300.mps import MPS, MPSError, MPS_ERR_ARG
    m = MPS(4, 4, 0.0)
    with pytest.raises(MPSError) as e:
        m.sample(np.array([[0.1, 0.2, 1.0, 0.3]]))
    assert e.value.code == MPS_ERR_ARG
    with pytest.raises(MPSError) as e:
        m.pauli_expectations(["XYQZ"])
    assert e.value.code == MPS_ERR_ARG
