"""The randomized-sketch SVD path (MPS_SVD_SKETCH_MLP) through the C ABI:
whatever the predictor says, the results equal the oracle's full-SVD
results within the binary64 tolerances (an accepted sketch captured the
spectrum above the threshold; a rejected one fell back to the full SVD)."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1111_3124_gb300 import circuits as C
from tests.helpers import random_state, spectrum_err, two_site_tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    t.cuda.set_device(0)
    from paper_1111_3124_gb300 import build as B
    B.build()
    from paper_1111_3124_gb300 import mps
    return mps


def constant_predictor(M, rank):
    """An MLP whose output is the constant log2(rank)/10 (all weights zero)."""
    m = M.RankPredictor(seed=0)
    p = np.zeros(M.MLP_PARAMS, dtype=np.float32)
    p[mlp.B2] = np.log2(rank) / 10.0
    m.params = p
    return m


def run(M, n, layers, chi_max, cutoff, pred, prec=0):
    g = M.MPS(n, chi_max, cutoff, prec)
    g.set_predictor(pred)
    g.set_mode(prec, 0, M.SVD_SKETCH_MLP)
    g.run_layers(layers)
    return g


def compare(g, n, layers, chi_max, cutoff):
    ref = oracle.OracleMPS(n, chi_max, cutoff)
    for layer in layers:
        for s, U in layer:
            ref.apply_gate(s, U)
    for b in range(n - 1):
        assert spectrum_err(g.schmidt(b), ref.schmidt(b)) < 1e-12
    bits = np.random.default_rng(3).integers(0, 2, size=(48, n)).astype(np.uint8)
    assert np.max(np.abs(g.amplitudes(bits) - np.array([ref.amplitude(b) for b in bits]))) < 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_sketch_accepted_when_rank_fits(M, prec):
    """Bonds (64, 20, 64) make theta 128 x 128 of rank <= 4 * 20 = 80 (a U(4)
    has operator-Schmidt rank <= 4): a predicted rank of 75 sizes a sketch of
    width 93, which captures theta exactly and is accepted; the update equals
    the oracle's full-SVD update."""
    chi = (1, 64, 20, 64, 1)
    n = len(chi) - 1
    state = random_state(n, chi, 31)
    U = C.haar_unitary(4, np.random.default_rng(32))
    ref = oracle.OracleMPS(n, 128, 1e-12)
    ref.set_state(*state)
    ref.apply_gate(1, U)
    g = M.MPS(n, 128, 1e-12, prec)
    g.import_state(*state)
    g.set_predictor(constant_predictor(M, 75))
    g.set_mode(prec, 0, M.SVD_SKETCH_MLP)
    g.apply_gate(1, U)
    st = g.sketch_stats()
    assert st["sketched"] == 1 and st["accepted"] == 1, st
    _, rg, rl = ref.get_state()
    _, gg, gl = g.export()
    assert len(gl[1]) == len(rl[1]) == 80
    assert spectrum_err(gl[1], rl[1]) < 1e-12
    tg, tr = two_site_tensor(gg, gl, 1), two_site_tensor(rg, rl, 1)
    assert np.max(np.abs(tg - tr)) < 1e-11 * np.max(np.abs(tr))


def test_diag_reports_kept_and_sketch_ranks(M):
    """mps_diag's k and k_sketch equal the counts of the oracle's singular
    values of the gate-applied theta above max(cutoff, Mw eps) ||sigma|| and
    max(cutoff/100, Mw eps) ||sigma|| (Sec. 3.1 truncation)."""
    chi = (1, 24, 40, 24, 1)
    n, cutoff = len(chi) - 1, 1e-3
    state = random_state(n, chi, 43)
    U = C.haar_unitary(4, np.random.default_rng(44))
    g = M.MPS(n, 128, cutoff, 0)
    g.import_state(*state)
    g.apply_gate(1, U)
    d = g.diag()
    gam, lam = state
    t = two_site_tensor(gam, lam, 1).reshape(2, chi[1], 2, chi[3])
    t2 = np.einsum("ijkl,kalb->iajb", U.reshape(2, 2, 2, 2), t).reshape(2 * chi[1], 2 * chi[3])
    sigma = oracle.svd(t2)[0]
    norm = np.sqrt(np.sum(sigma ** 2))
    mw_eps = max(t2.shape) * 2.0 ** -53
    thr_k, thr_sk = max(cutoff, mw_eps) * norm, max(cutoff / 100, mw_eps) * norm
    for thr in (thr_k, thr_sk):  # no value so close to a threshold that rounding decides it
        assert np.min(np.abs(sigma - thr)) > 1e-6 * thr
    assert int(np.sum(sigma > thr_k)) < int(np.sum(sigma > thr_sk)) < min(t2.shape)
    assert d["k"][0] == int(np.sum(sigma > thr_k))
    assert d["k_sketch"][0] == int(np.sum(sigma > thr_sk))


def test_sketch_falls_back_when_rank_too_small(M):
    n, chi_max, cutoff = 12, 32, 1e-12
    layers = C.brickwork(n, 8, np.random.default_rng(22))
    g = run(M, n, layers, chi_max, cutoff, constant_predictor(M, 2))
    st = g.sketch_stats()
    assert st["sketched"] > 0 and st["accepted"] < st["sketched"], st
    compare(g, n, layers, chi_max, cutoff)


def test_sketch_routes_full_rank_predictions_to_jacobi(M):
    n, chi_max, cutoff = 10, 16, 1e-12
    layers = C.brickwork(n, 6, np.random.default_rng(23))
    g = run(M, n, layers, chi_max, cutoff, constant_predictor(M, 1000))
    st = g.sketch_stats()
    assert st["sketched"] == 0 and st["routed_full"] > 0, st
    compare(g, n, layers, chi_max, cutoff)
