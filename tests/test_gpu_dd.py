"""The double-word (about 106-bit) GPU path (mps_dd_*) against the oracle in
binary128, on circuits whose gates are unitary to ~1e-32 (hi + lo inputs).

Tolerances. A double-word operation has relative error <= 5u^2 (u = 2^-53,
u^2 ~ 1.2e-32); one update's results carry ~mw u^2 relative error (mw <= 64
rows of the Jacobi working matrix) amplified by the conditioning of the
Lambda^-1 rewrite; over a few dozen updates this stays below 1e-27 relative
to the largest value, against ~1e-14 for the binary64 path on the same
inputs (printed beside it)."""
import numpy as np
import pytest

import oracle
from paper_1111_3124_gb300 import circuits as C
from tests.helpers import all_bits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1111_3124_gb300 import build as B
    B.build()


def _run_dd(n, layers, chi, cutoff):
    from paper_1111_3124_gb300.mps import MPSDD
    m = MPSDD(n, chi, cutoff)
    for layer in layers:
        by_d = {}
        for site, Uh, Ul in layer:
            by_d.setdefault(Uh.shape[0], []).append((site, Uh, Ul))
        for d in sorted(by_d):
            g = by_d[d]
            m.apply_layer([s for s, _, _ in g], np.stack([u for _, u, _ in g]), np.stack([l for _, _, l in g]))
    m.sync()
    return m


def _run_oracle(n, layers, chi, cutoff):
    o = oracle.OracleMPS(n, chi, cutoff, oracle.BINARY128)
    for layer in layers:
        for site, Uh, Ul in layer:
            o.apply_gate_hl(site, Uh, Ul)
    return o


def _dd_diff(a_hi, a_lo, b_hi, b_lo):
    """|(a_hi + a_lo) - (b_hi + b_lo)| without losing the low parts."""
    return np.abs((np.asarray(a_hi) - np.asarray(b_hi)) + (np.asarray(a_lo) - np.asarray(b_lo)))


def _compare(m, o, n, bits, tol):
    worst_s = 0.0
    for b in range(n - 1):
        hi, lo = m.schmidt(b)
        ohi, olo = o.schmidt_hl(b)
        assert len(hi) == len(ohi), (b, len(hi), len(ohi))
        worst_s = max(worst_s, float(np.max(_dd_diff(hi, lo, ohi, olo)) / ohi[0]))
    amps = m.amplitudes(bits)
    ref = np.array([o.amplitude_hl(b) for b in bits])
    scale = float(np.max(np.abs(ref[:, 0] + 1j * ref[:, 2])))
    d_re = _dd_diff(amps[:, 0], amps[:, 1], ref[:, 0], ref[:, 1])
    d_im = _dd_diff(amps[:, 2], amps[:, 3], ref[:, 2], ref[:, 3])
    worst_a = float(np.max(np.hypot(d_re, d_im)) / scale)
    assert worst_s < tol and worst_a < tol, (worst_s, worst_a)
    return worst_s, worst_a


def test_dd_ghz_spectrum_closed_form():
    n = 16
    m = _run_dd(n, C.dd_ghz_prefix(n), 4, 1e-28)
    from decimal import Decimal, localcontext
    with localcontext() as ctx:
        ctx.prec = 60
        r = Decimal(1) / Decimal(2).sqrt()
        r_hi = float(r)
        r_lo = float(r - Decimal(r_hi))  # 1/sqrt(2) as hi + lo
    for b in range(n - 1):
        hi, lo = m.schmidt(b)
        assert len(hi) == 2
        assert np.max(_dd_diff(hi, lo, [r_hi] * 2, [r_lo] * 2)) < 1e-31
    a = m.amplitudes(np.ones((1, n), dtype=np.uint8))[0]
    assert abs((a[0] - r_hi) + (a[1] - r_lo)) < 1e-31 and abs(a[2]) + abs(a[3]) < 1e-31
    m.close()


def test_dd_exact_circuit_all_amplitudes_vs_binary128_oracle():
    """n = 10, chi_max = 32: nothing is truncated; all 1024 amplitudes."""
    n, chi, cutoff = 10, 32, 1e-28
    layers = C.dd_brickwork(n, 8, np.random.default_rng(9001))
    m = _run_dd(n, layers, chi, cutoff)
    o = _run_oracle(n, layers, chi, cutoff)
    ws, wa = _compare(m, o, n, all_bits(n), 1e-28)
    print("exact circuit: spectrum err %.2e, amplitude err %.2e" % (ws, wa))
    assert m.bond_dims().max() == 32
    st = m.stats()
    assert st["updates"] == C.count_updates([[(s, U) for s, U, _ in l] for l in layers])
    assert st["flops"] > 0 and st["sweeps"] > 0
    m.close()


def test_dd_truncating_circuit_vs_binary128_oracle_and_binary64():
    n, chi, cutoff = 14, 8, 1e-28
    layers = C.dd_brickwork(n, 8, np.random.default_rng(9002))
    m = _run_dd(n, layers, chi, cutoff)
    o = _run_oracle(n, layers, chi, cutoff)
    bits = np.random.default_rng(1).integers(0, 2, size=(128, n)).astype(np.uint8)
    ws, wa = _compare(m, o, n, bits, 1e-26)
    # the binary64 GPU path on the same gates (hi parts only): ~1e-14
    from paper_1111_3124_gb300.mps import MPS
    m64 = MPS(n, chi, cutoff)
    m64.run_layers([[(s, Uh) for s, Uh, _ in l] for l in layers])
    e64 = max(float(np.max(np.abs(m64.schmidt(b) - (o.schmidt_hl(b)[0] + o.schmidt_hl(b)[1]))))
              for b in range(n - 1))
    print("truncating circuit: double-word spectrum err %.2e, amplitude err %.2e; binary64 spectrum err %.2e"
          % (ws, wa, e64))
    assert e64 > 1e3 * ws
    m.close()
    m64.close()


def test_dd_single_site_gates_and_layer_checks():
    from paper_1111_3124_gb300.mps import MPSDD, MPSError, MPS_ERR_ARG, MPS_ERR_TOO_LARGE
    n = 6
    rng = np.random.default_rng(5)
    layers = [[(q,) + C.dd_unitary(C.haar_unitary(2, rng)) for q in range(n)]] + C.dd_brickwork(n, 3, rng)
    m = _run_dd(n, layers, 8, 1e-28)
    o = _run_oracle(n, layers, 8, 1e-28)
    _compare(m, o, n, all_bits(n), 1e-28)
    with pytest.raises(MPSError) as e:
        m.apply_layer([0, 1], np.stack([C.CNOT, C.CNOT]))  # overlapping gates
    assert e.value.code == MPS_ERR_ARG
    with pytest.raises(MPSError) as e:
        m.apply_layer([5], np.stack([C.CNOT]))  # past the last qubit
    assert e.value.code == MPS_ERR_ARG
    with pytest.raises(MPSError) as e:
        MPSDD(8, 33, 1e-28)
    assert e.value.code == MPS_ERR_TOO_LARGE
    m.close()


def test_dd_sweep_limit_reports_noconverge_and_leaves_the_gate_unapplied():
    from paper_1111_3124_gb300.mps import MPSError, MPS_ERR_NOCONVERGE
    n = 8
    layers = C.dd_brickwork(n, 4, np.random.default_rng(6))
    m = _run_dd(n, layers, 16, 1e-28)
    before = m.amplitudes(all_bits(n))
    m.set_limits(1)
    g = C.dd_unitary(C.haar_unitary(4, np.random.default_rng(7)))
    m.apply_layer([3], g[0][None], g[1][None])
    with pytest.raises(MPSError) as e:
        m.sync()
    assert e.value.code == MPS_ERR_NOCONVERGE
    assert np.array_equal(m.amplitudes(all_bits(n)), before)
    m.close()
