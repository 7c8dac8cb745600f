"""Many independent circuits of mixed size and chi_max updated in shared
batched passes (mps_apply_layer_multi), against each circuit run alone and
against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1111_3124_gb300 import circuits as C
from tests.helpers import spectrum_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    t.cuda.set_device(0)
    from paper_1111_3124_gb300 import build as B
    B.build()
    return t


def _specs():
    # (n, depth, chi_max): mixed sizes, some truncating, small enough for the oracle
    return [(6, 5, 4), (9, 6, 8), (12, 7, 16), (7, 4, 64), (10, 8, 6), (16, 6, 32)]


@pytest.mark.parametrize("prec", [0, 1])
def test_multi_circuit_batch_matches_oracle(torch, prec):
    from paper_1111_3124_gb300.mps import MPS, apply_layer_multi
    specs = _specs()
    circuits = [C.brickwork(n, d, np.random.default_rng(500 + i), first_u2_layer=True) for i, (n, d, _) in enumerate(specs)]
    states = [MPS(n, chi, 1e-12, prec) for (n, _, chi) in specs]
    depth = max(len(c) for c in circuits)
    for l in range(depth):
        per_state_1q, per_state_2q = [], []
        for c in circuits:
            layer = c[l] if l < len(c) else []
            per_state_1q.append([(s, U) for s, U in layer if U.shape[0] == 2])
            per_state_2q.append([(s, U) for s, U in layer if U.shape[0] == 4])
        for m, layer in zip(states, per_state_1q):
            if layer:
                m.apply_layer([s for s, _ in layer], np.stack([U for _, U in layer]))
        apply_layer_multi(states, per_state_2q)
    rng = np.random.default_rng(7)
    for (n, _, chi), c, m in zip(specs, circuits, states):
        ref = oracle.OracleMPS(n, chi, 1e-12)
        for layer in c:
            for s, U in layer:
                ref.apply_gate(s, U)
        for b in range(n - 1):
            assert spectrum_err(m.schmidt(b), ref.schmidt(b)) < 1e-12
        bits = rng.integers(0, 2, size=(32, n)).astype(np.uint8)
        a = m.amplitudes(bits)
        assert np.max(np.abs(a - np.array([ref.amplitude(x) for x in bits]))) < 1e-10


def test_multi_rejects_bad_input_and_applies_nothing(torch):
    from paper_1111_3124_gb300.mps import MPS, MPSError, apply_layer_multi
    a, b = MPS(4, 8, 0.0), MPS(5, 8, 0.0)
    with pytest.raises(MPSError):
        apply_layer_multi([a, b], [[(0, C.CNOT)], [(4, C.CNOT)]])  # site 4 out of range for n = 5
    with pytest.raises(MPSError):
        apply_layer_multi([a, b], [[(0, 2 * np.eye(4))], [(0, C.CNOT)]])  # not unitary
    assert abs(a.amplitude([0, 0, 0, 0]) - 1) < 1e-15 and abs(b.amplitude([0] * 5) - 1) < 1e-15
