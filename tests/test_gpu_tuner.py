"""Every launch shape the tuner chooses between gives the oracle's result, and
the tuner's table round-trips through its cache."""
import numpy as np
import pytest

import oracle
from paper_1111_3124_gb300 import circuits as C
from tests.helpers import spectrum_err, two_site_tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1111_3124_gb300 import build as B
    B.build()


@pytest.mark.parametrize("cand", [(16, 3), (8, 3), (16, 2), (8, 2), (16, 0), (8, 0), (16, 1)])
def test_every_candidate_matches_the_oracle(cand):
    from paper_1111_3124_gb300.mps import MPS, PREC_SPLIT
    # a saturated update, theta 128 x 128 cut to 64
    rng = np.random.default_rng(600 + cand[0] + cand[1])
    state = C.random_vidal_state(4, (1, 64, 64, 64, 1), rng, decay=2.0)
    U = C.haar_unitary(4, rng)
    orc = oracle.OracleMPS(4, 64, 1e-12)
    orc.set_state(*state)
    orc.apply_gate(1, U)
    m = MPS(4, 64, 1e-12, PREC_SPLIT)
    m.set_tuning([(4096, cand[0], cand[1])])
    m.import_state(*state)
    m.apply_gate(1, U)
    _, og, ol = orc.get_state()
    _, gg, gl = m.export()
    assert spectrum_err(gl[1], ol[1]) < 1e-12
    t_o, t_g = two_site_tensor(og, ol, 1), two_site_tensor(gg, gl, 1)
    assert np.max(np.abs(t_o - t_g)) < 1e-11 * np.max(np.abs(t_o))
    # and a truncating circuit from |0...0>
    n, chi_max = 12, 16
    layers = C.brickwork(n, 8, rng)
    g = MPS(n, chi_max, 1e-12, PREC_SPLIT)
    g.set_tuning([(4096, cand[0], cand[1])])
    g.run_layers(layers)
    o = oracle.OracleMPS(n, chi_max, 1e-12)
    for layer in layers:
        for site, V in layer:
            o.apply_gate(site, V)
    for b in range(n - 1):
        assert spectrum_err(g.schmidt(b), o.schmidt(b)) < 1e-12


def test_tuning_table_rejects_bad_entries():
    from paper_1111_3124_gb300.mps import MPS, MPSError, MPS_ERR_ARG
    m = MPS(4, 8, 0.0)
    for table in ([(64, 12, 0)], [(64, 8, 1)], [(64, 16, 4)], [(64, 16, -1)], [(128, 16, 0), (64, 16, 0)]):
        with pytest.raises(MPSError) as e:
            m.set_tuning(table)
        assert e.value.code == MPS_ERR_ARG
    m.set_tuning([])


def test_tuner_picks_a_candidate_and_caches_it(tmp_path):
    from paper_1111_3124_gb300 import tuner
    table, meas = tuner.tune(chis=(16, 32), reps=1, n=16)
    assert [r[0] for r in table] == [32, 64]
    for nw, bw, mode in table:
        assert (bw, mode) in tuner.CANDIDATES
        assert len(meas[str(nw)]) == len(tuner.CANDIDATES)
    path = tuner.save(table, meas, str(tmp_path / "tune.json"))
    assert tuner.load(path) == [tuple(r) for r in table]
