"""Recorded circuits (mps_program_*): the gate updates of a whole circuit, or
of many circuits at once, replayed as one CUDA graph whose Jacobi sweep loops
are conditional nodes controlled on the device. Checked against the state
vector, the oracle and the eager (host-driven) path on the same inputs."""
import numpy as np
import pytest

import oracle
from oracle.statevector import StateVector
from paper_1111_3124_gb300 import circuits as C
from tests.helpers import all_bits, spectrum_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1111_3124_gb300 import build as B
    B.build()


def _statevector(n, layers):
    sv = StateVector(n)
    for layer in layers:
        for site, U in layer:
            k = {2: 1, 4: 2, 8: 3}[U.shape[0]]
            sv.apply(list(range(site, site + k)), U)
    return sv


def _oracle(n, layers, chi_max, cutoff):
    m = oracle.OracleMPS(n, chi_max, cutoff)
    for layer in layers:
        for site, U in layer:
            m.apply_gate(site, U)
    return m


@pytest.mark.parametrize("prec", [0, 1])
def test_program_n10_brickwork_all_amplitudes(prec):
    from paper_1111_3124_gb300.mps import MPS, Program, circuit_passes
    c = C.WORKLOADS[C.N10]
    n = c["n"]
    layers = C.workload_circuit(C.N10)
    m = MPS(n, c["chi_max"], c["cutoff"], prec)
    prog = Program([m], circuit_passes(layers))
    assert prog.updates == C.count_updates(layers)
    prog.run()
    amps = m.amplitudes(all_bits(n))
    assert np.max(np.abs(amps - _statevector(n, layers).vector())) < 1e-10
    # replayed from |0...0> it gives the same state again
    m.reset()
    prog.run()
    assert np.max(np.abs(m.amplitudes(all_bits(n)) - amps)) < 1e-14
    prog.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_program_truncating_circuit_vs_oracle_and_eager(prec):
    from paper_1111_3124_gb300.mps import MPS, Program, circuit_passes
    rng = np.random.default_rng(5150)
    n, chi_max, cutoff = 14, 12, 1e-12
    layers = C.brickwork(n, 10, rng, rz_after_each=True)
    m = MPS(n, chi_max, cutoff, prec)
    prog = Program([m], circuit_passes(layers))
    prog.run()
    eager = MPS(n, chi_max, cutoff, prec)
    eager.run_layers(layers)
    orc = _oracle(n, layers, chi_max, cutoff)
    bits = np.random.default_rng(3).integers(0, 2, size=(128, n)).astype(np.uint8)
    a = m.amplitudes(bits)
    assert np.max(np.abs(a - eager.amplitudes(bits))) < 1e-12
    assert np.max(np.abs(a - np.array([orc.amplitude(b) for b in bits]))) < 1e-10
    for b in range(n - 1):
        assert spectrum_err(m.schmidt(b), orc.schmidt(b)) < 1e-12
    prog.close()


def test_program_three_site_gates_vs_oracle():
    from paper_1111_3124_gb300.mps import MPS, Program, circuit_passes
    rng = np.random.default_rng(77)
    n, chi_max, cutoff = 12, 16, 1e-12
    layers = C.ghz_prefix(n) + C.u8_shifted_brick(n, 4, rng)
    for prec in (0, 1):
        m = MPS(n, chi_max, cutoff, prec)
        prog = Program([m], circuit_passes(layers))
        prog.run()
        orc = _oracle(n, layers, chi_max, cutoff)
        bits = np.random.default_rng(4).integers(0, 2, size=(64, n)).astype(np.uint8)
        assert np.max(np.abs(m.amplitudes(bits) - np.array([orc.amplitude(b) for b in bits]))) < 1e-10
        for b in range(n - 1):
            assert spectrum_err(m.schmidt(b), orc.schmidt(b)) < 1e-12
        prog.close()


def test_program_many_circuits_in_shared_passes():
    """Circuits of different n, depth and chi_max, recorded as passes that hold
    the depth-d layer of every circuit (the batched workload), against each
    circuit run alone on the eager path."""
    import torch
    from paper_1111_3124_gb300.mps import MPS, Program
    rng = np.random.default_rng(808)
    specs = [(10, 5, 8), (14, 7, 16), (12, 3, 32), (9, 6, 4)]
    circuits = [C.brickwork(n, d, rng) for n, d, _ in specs]
    states = [MPS(n, chi, 1e-12, 1) for n, _, chi in specs]
    passes = []
    for depth in range(max(d for _, d, _ in specs)):
        for kq, dim in ((1, 2), (2, 4)):
            gates, mats = [], []
            for i, layers in enumerate(circuits):
                if depth < len(layers):
                    for site, U in layers[depth]:
                        if U.shape[0] == dim:
                            gates.append((i, site))
                            mats.append(U)
            if gates:
                passes.append((kq, gates, torch.from_numpy(np.stack(mats).astype(np.complex128)).cuda()))
    prog = Program(states, passes)
    prog.run()
    for (n, _, chi), layers, m in zip(specs, circuits, states):
        ref = MPS(n, chi, 1e-12, 1)
        ref.run_layers(layers)
        bits = np.random.default_rng(n).integers(0, 2, size=(64, n)).astype(np.uint8)
        assert np.max(np.abs(m.amplitudes(bits) - ref.amplitudes(bits))) < 1e-12
    prog.close()


def test_program_refuses_a_state_above_its_bounds():
    from paper_1111_3124_gb300.mps import MPS, MPSError, MPS_ERR_ARG, Program, circuit_passes
    rng = np.random.default_rng(9)
    n = 8
    layers = C.brickwork(n, 2, rng)
    m = MPS(n, 16, 1e-12)
    prog = Program([m], circuit_passes(layers))
    m.run_layers(C.brickwork(n, 3, rng))  # bonds now above the recorded |0...0> bounds
    with pytest.raises(MPSError) as e:
        prog.run()
    assert e.value.code == MPS_ERR_ARG
    m.reset()
    prog.run()
    m.sync()
    prog.close()


def test_program_sweep_limit_reports_noconverge():
    """The sweep loop of a replay stops at the limit on the device and the
    status reaches the host at the next synchronising call."""
    from paper_1111_3124_gb300.mps import MPS, MPSError, MPS_ERR_NOCONVERGE, Program, circuit_passes
    rng = np.random.default_rng(10)
    n = 8
    m = MPS(n, 16, 1e-12)
    m.set_limits(1)
    prog = Program([m], circuit_passes(C.brickwork(n, 4, rng)))
    prog.run()
    with pytest.raises(MPSError) as e:
        m.sync()
    assert e.value.code == MPS_ERR_NOCONVERGE
    prog.close()
