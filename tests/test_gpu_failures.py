"""Failure paths of the C ABI on the GPU, made on the host side (no GPU fault,
trap or hang is ever provoked):

  * MPS_ERR_NOCONVERGE: the binary64 Jacobi sweep limit set to 1, so a gate
    whose SVD needs more sweeps stops at the limit; the gate is left
    unapplied (tensors byte-identical) and the next synchronising call
    reports the status;
  * MPS_ERR_NOMEM: the library's allocation hook refuses an allocation, at
    handle creation and when a wider layer needs a larger workspace; the call
    fails synchronously and leaves the state (and its held-back single-qubit
    gates) as it was.

A timeout of the split GEMM's bounded waits is not provoked on the GPU:
forcing one would abandon tensor-core products and copies in flight. The
handle treats such a timeout as sticky (every later split-precision product
is refused), which is host logic only.
"""
import numpy as np
import pytest

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


def _state_bytes(m):
    chi, gammas, lams = m.export()
    return chi.tobytes() + b"".join(g.tobytes() for g in gammas) + b"".join(l.tobytes() for l in lams)


def _entangled(n, chi_max, seed, prec=0):
    from paper_1111_3124_gb300.mps import MPS
    rng = np.random.default_rng(seed)
    m = MPS(n, chi_max, 1e-12, prec)
    m.run_layers(C.brickwork(n, 4, rng))
    return m, rng


def test_sweep_limit_reports_noconverge_and_leaves_the_gate_unapplied():
    from paper_1111_3124_gb300.mps import MPSError, MPS_ERR_NOCONVERGE
    m, rng = _entangled(8, 16, 11)
    before = _state_bytes(m)
    m.set_limits(1)
    U = C.haar_unitary(4, rng)
    m.apply_gate(3, U)  # asynchronous: the status is deferred
    with pytest.raises(MPSError) as e:
        m.sync()
    assert e.value.code == MPS_ERR_NOCONVERGE
    assert _state_bytes(m) == before
    m.sync()  # the status was cleared by the report
    # with the default limit the same gate applies and matches a fresh handle
    m.set_limits(60)
    m.apply_gate(3, U)
    m.sync()
    ref, _ = _entangled(8, 16, 11)
    ref.apply_gate(3, U)
    a = m.amplitudes(np.eye(8, dtype=np.uint8))
    b = ref.amplitudes(np.eye(8, dtype=np.uint8))
    assert np.max(np.abs(a - b)) < 1e-13


def test_sweep_limit_argument_range():
    from paper_1111_3124_gb300.mps import MPS, MPSError, MPS_ERR_ARG
    m = MPS(4, 8, 0.0)
    for bad in (0, 61, -3):
        with pytest.raises(MPSError) as e:
            m.set_limits(bad)
        assert e.value.code == MPS_ERR_ARG


def test_refused_allocation_at_creation():
    from paper_1111_3124_gb300.mps import MPS, MPSError, MPS_ERR_NOMEM, debug_fail_alloc
    for after in (0, 1, 2):
        debug_fail_alloc(after)
        try:
            with pytest.raises(MPSError) as e:
                MPS(6, 8, 0.0)
            assert e.value.code == MPS_ERR_NOMEM
        finally:
            debug_fail_alloc(-1)
    MPS(6, 8, 0.0).close()  # the hook is off again


@pytest.mark.parametrize("prec", [0, 1])
def test_refused_workspace_growth_keeps_state_and_held_back_gates(prec):
    from paper_1111_3124_gb300.mps import MPS, MPSError, MPS_ERR_NOMEM, debug_fail_alloc
    n = 10
    rng = np.random.default_rng(23)
    small = C.haar_unitary(4, rng)
    h1 = C.haar_unitary(2, rng)
    wide = [C.haar_unitary(4, rng) for _ in range(n // 2)]
    sites = list(range(0, n, 2))

    def prefix(m):
        m.apply_gate(0, small)       # a one-gate pass: a small workspace
        m.apply_gate(2, h1)          # held back, folded into the next gate on qubit 2

    m = MPS(n, 32, 1e-12, prec)
    prefix(m)
    m.sync()
    chi_before = m.bond_dims().copy()
    debug_fail_alloc(0)
    try:
        with pytest.raises(MPSError) as e:
            m.apply_layer(sites, np.stack(wide))  # five gates: the workspace must grow
        assert e.value.code == MPS_ERR_NOMEM
    finally:
        debug_fail_alloc(-1)
    assert np.array_equal(m.bond_dims(), chi_before)
    m.apply_layer(sites, np.stack(wide))  # retried: the held-back gate on qubit 2 is still applied once
    ref = MPS(n, 32, 1e-12, prec)
    prefix(ref)
    ref.apply_layer(sites, np.stack(wide))
    bits = np.random.default_rng(5).integers(0, 2, size=(64, n)).astype(np.uint8)
    assert np.max(np.abs(m.amplitudes(bits) - ref.amplitudes(bits))) < 1e-13


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    """The tensor-core kernels' bounded mbarrier wait, on a barrier nothing
    completes, gives up after its limit and reports MPS_ERR_TIMEOUT; nothing
    was in flight, so a split-precision update right after it is unaffected."""
    from paper_1111_3124_gb300.mps import (MPS, MPSError, MPS_ERR_TIMEOUT, PREC_SPLIT, debug_bounded_wait)
    import time
    t0 = time.perf_counter()
    with pytest.raises(MPSError) as e:
        debug_bounded_wait(5.0)
    assert e.value.code == MPS_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    n = 8
    layers = C.brickwork(n, 4, np.random.default_rng(31))
    a = MPS(n, 16, 1e-12, PREC_SPLIT)
    a.run_layers(layers)
    b = MPS(n, 16, 1e-12)
    b.run_layers(layers)
    bits = np.random.default_rng(2).integers(0, 2, size=(32, n)).astype(np.uint8)
    assert np.max(np.abs(a.amplitudes(bits) - b.amplitudes(bits))) < 1e-12
    a.close()
    b.close()


def test_a_timed_out_handle_refuses_split_products_and_keeps_its_state():
    """After a timeout of its split GEMM (marked here on the host: forcing one
    on the GPU would abandon copies and products in flight), a handle refuses
    every later split-precision update with MPS_ERR_TIMEOUT before launching
    anything: its tensors stay as they were."""
    from paper_1111_3124_gb300.mps import MPS, MPSError, MPS_ERR_TIMEOUT, PREC_SPLIT, debug_mark_timed_out
    n = 8
    m = MPS(n, 16, 1e-12, PREC_SPLIT)
    m.run_layers(C.brickwork(n, 3, np.random.default_rng(32)))
    bits = np.random.default_rng(3).integers(0, 2, size=(32, n)).astype(np.uint8)
    before = m.amplitudes(bits)
    debug_mark_timed_out(m)
    for _ in range(2):
        with pytest.raises(MPSError) as e:
            m.apply_layer([2], C.haar_unitary(4, np.random.default_rng(4))[None])
        assert e.value.code == MPS_ERR_TIMEOUT
    assert np.array_equal(m.amplitudes(bits), before)
    m.close()
