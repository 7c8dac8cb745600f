"""The scheduled fp32 sweeps (every sweep of every task of a pass in one
launch, block pairs taken in order as their inputs become final) against one
launch per round-robin round. Both run the same rotations on the same data, so
the states must agree bit for bit: eagerly, in recorded programs, for U(8)
gates and for passes that mix widths and circuits. The oracle checks the
scheduled result on its own as well, and the 384-thread form of the scheduled
launch, whose Grams sum their rows in another grouping."""
import numpy as np
import pytest

import oracle
from paper_1111_3124_gb300 import circuits as C
from tests.helpers import spectrum_err

pytestmark = pytest.mark.gpu

ROUND, SCHED, SCHED384 = 0, 2, 3  # launch modes of mps_set_tuning


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1111_3124_gb300 import build as B
    B.build()


def _same(a, b):
    chi_a, g_a, l_a = a
    chi_b, g_b, l_b = b
    assert np.array_equal(chi_a, chi_b)
    for x, y in zip(g_a, g_b):
        assert np.array_equal(x, y)
    for x, y in zip(l_a, l_b):
        assert np.array_equal(x, y)


def _saturated_state(n, chi, rng):
    chis = [1] + [min(chi, 2 ** min(b, n - b)) for b in range(1, n)] + [1]
    return C.random_vidal_state(n, chis, rng, decay=2.0)


def _run_eager(n, chi, table, layers, state=None):
    from paper_1111_3124_gb300.mps import MPS, PREC_SPLIT
    m = MPS(n, chi, 1e-12, PREC_SPLIT)
    try:
        m.set_tuning(table)
        if state is not None:
            m.import_state(*state)
        m.run_layers(layers)
        return m.export(), m.diag()
    finally:
        m.close()


@pytest.mark.parametrize("bw", [16, 8])
def test_saturated_layers_bit_for_bit(bw):
    rng = np.random.default_rng(910 + bw)
    n, chi = 16, 64
    state = _saturated_state(n, chi, rng)
    layers = [[(s, C.haar_unitary(4, rng)) for s in C.brickwork_sites(n, p)] for p in (0, 1, 0)]
    a, da = _run_eager(n, chi, [(4096, bw, ROUND)], layers, state)
    b, db = _run_eager(n, chi, [(4096, bw, SCHED)], layers, state)
    _same(a, b)
    for key in ("k", "sweeps", "discarded"):
        assert np.array_equal(da[key], db[key])
    # and the scheduled result against the oracle
    o = oracle.OracleMPS(n, chi, 1e-12)
    o.set_state(*state)
    for layer in layers:
        for s, U in layer:
            o.apply_gate(s, U)
    for bnd in range(n - 1):
        assert spectrum_err(b[2][bnd], o.schmidt(bnd)) < 1e-12


def test_truncating_circuit_from_zero_bit_for_bit():
    # bonds grow from 1 and are cut at chi_max: every pass mixes widths
    rng = np.random.default_rng(920)
    n, chi = 14, 24
    layers = C.brickwork(n, 10, rng, first_u2_layer=True)
    a, _ = _run_eager(n, chi, [(4096, 16, ROUND)], layers)
    b, _ = _run_eager(n, chi, [(4096, 16, SCHED)], layers)
    _same(a, b)


def test_three_site_gates_bit_for_bit():
    rng = np.random.default_rng(930)
    n, chi = 12, 32
    layers = [[(s, C.haar_unitary(8, rng)) for s in range(p, n - 2, 3)] for p in (0, 1, 2, 0)]
    a, _ = _run_eager(n, chi, [(4096, 16, ROUND)], layers)
    b, _ = _run_eager(n, chi, [(4096, 16, SCHED)], layers)
    _same(a, b)


def _run_program(n, chi, table, layers, replays):
    from paper_1111_3124_gb300.mps import MPS, PREC_SPLIT, Program, circuit_passes
    m = MPS(n, chi, 1e-12, PREC_SPLIT)
    prog = None
    try:
        m.set_tuning(table)
        prog = Program([m], circuit_passes(layers))
        outs = []
        for _ in range(replays):
            m.reset()
            prog.run()
            m.sync()
            outs.append(m.export())
        return outs
    finally:
        if prog is not None:
            prog.close()
        m.close()


def test_recorded_programs_bit_for_bit():
    # one CUDA graph per circuit; the scheduled launch is one graph node per pass
    rng = np.random.default_rng(940)
    n, chi = 16, 32
    layers = C.brickwork(n, 12, rng, first_u2_layer=True)
    a = _run_program(n, chi, [(4096, 16, ROUND)], layers, 1)
    b = _run_program(n, chi, [(4096, 16, SCHED)], layers, 2)
    _same(a[0], b[0])
    _same(b[0], b[1])  # a replay after reset gives the same state again


def test_many_circuits_of_mixed_size_in_shared_passes():
    from paper_1111_3124_gb300.mps import MPS, PREC_SPLIT, apply_layer_multi
    specs = [(6, 5, 4), (9, 6, 8), (12, 7, 16), (16, 6, 32), (10, 8, 64)]
    circuits = [C.brickwork(n, d, np.random.default_rng(950 + i)) for i, (n, d, _) in enumerate(specs)]
    results = {}
    for mode in (ROUND, SCHED):
        states = [MPS(n, chi, 1e-12, PREC_SPLIT) for (n, _, chi) in specs]
        try:
            for m in states:
                m.set_tuning([(4096, 16, mode)])
            for l in range(max(len(c) for c in circuits)):
                apply_layer_multi(states, [c[l] if l < len(c) else [] for c in circuits])
            results[mode] = [m.export() for m in states]
        finally:
            for m in states:
                m.close()
    for a, b in zip(results[ROUND], results[SCHED]):
        _same(a, b)


@pytest.mark.parametrize("bw", [16, 8])
def test_384_thread_ctas_match_the_oracle(bw):
    rng = np.random.default_rng(960 + bw)
    n, chi = 16, 64
    state = _saturated_state(n, chi, rng)
    layers = [[(s, C.haar_unitary(4, rng)) for s in C.brickwork_sites(n, p)] for p in (0, 1, 0)]
    b, _ = _run_eager(n, chi, [(4096, bw, SCHED384)], layers, state)
    o = oracle.OracleMPS(n, chi, 1e-12)
    o.set_state(*state)
    for layer in layers:
        for s, U in layer:
            o.apply_gate(s, U)
    for bnd in range(n - 1):
        assert spectrum_err(b[2][bnd], o.schmidt(bnd)) < 1e-12
    # a truncating circuit from |0...0> and U(8) gates
    n2, chi2 = 14, 24
    layers2 = C.brickwork(n2, 10, rng, first_u2_layer=True)
    layers2 += [[(s, C.haar_unitary(8, rng)) for s in range(p, n2 - 2, 3)] for p in (0, 1)]
    c, _ = _run_eager(n2, chi2, [(4096, bw, SCHED384)], layers2)
    o2 = oracle.OracleMPS(n2, chi2, 1e-12)
    for layer in layers2:
        for s, U in layer:
            o2.apply_gate(s, U)
    for bnd in range(n2 - 1):
        assert spectrum_err(c[2][bnd], o2.schmidt(bnd)) < 1e-12
