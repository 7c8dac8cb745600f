"""The split-precision path (MPS_PREC_SPLIT) on the GPU, through the C ABI.

1. The tcgen05 split GEMM against numpy's binary64 product: error relative to
   |A||B| elementwise, per slice count, on random, ragged, zero and wide-
   exponent inputs.
2. Gate updates in split mode against the CPU oracle, with the tolerances of
   the binary64 path (amplitudes 1e-10 absolute, spectra 1e-12 lambda_0,
   reconstructed tensors 1e-11 of their largest entry).
"""
import numpy as np
import pytest

import oracle
from oracle.statevector import StateVector
from paper_1111_3124_gb300 import circuits as C
from tests.helpers import all_bits, oracle_run, random_state, spectrum_err, two_site_tensor

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


def _gemm_err(torch, m, n, k, slices=8, scale=None, seed=0, zero_rows=False):
    from paper_1111_3124_gb300.mps import split_zgemm
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
    B = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    if scale:
        A *= (2.0 ** rng.integers(-scale, scale, size=m))[:, None]
        B *= (2.0 ** rng.integers(-scale, scale, size=n))[None, :]
    if zero_rows:
        A[::3] = 0
        B[:, 1::4] = 0
    Cg = split_zgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), slices).cpu().numpy()
    bound = np.abs(A) @ np.abs(B)
    err = np.abs(Cg - A @ B)
    if zero_rows:
        assert np.all(Cg[::3] == 0) and np.all(Cg[:, 1::4] == 0)
    return float(np.max(err / np.where(bound > 0, bound, 1.0)))


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (5, 3, 7), (64, 64, 64), (200, 130, 77), (129, 65, 300), (512, 512, 512)])
def test_split_gemm_binary64_accuracy(torch, m, n, k):
    assert _gemm_err(torch, m, n, k) < 4e-15


def test_split_gemm_wide_exponents_and_zeros(torch):
    assert _gemm_err(torch, 256, 200, 256, scale=40, seed=3) < 4e-15
    assert _gemm_err(torch, 100, 90, 80, zero_rows=True, seed=5) < 4e-15


def test_split_gemm_error_falls_with_slices(torch):
    errs = [_gemm_err(torch, 150, 120, 100, slices=s, seed=9) for s in (2, 3, 4, 5, 6, 8)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[1] < 2e-5 and errs[3] < 2e-9


@pytest.mark.parametrize("k", [513, 1024, 1500])
def test_split_gemm_long_k_in_chunks(torch, k):
    assert _gemm_err(torch, 130, 70, k, seed=k) < 8e-15


@pytest.mark.parametrize("m,k", [(200, 130), (512, 700), (1024, 1300)])
def test_split_gram_is_exactly_hermitian(torch, m, k):
    # A^H A from conj(A)^T and A: every digit product is an exact integer and
    # the slice pairs are symmetric, so the product is Hermitian bit for bit.
    # The update's Gram and Newton-Schulz products rely on this: they multiply
    # the tiles on and above the diagonal and mirror them.
    from paper_1111_3124_gb300.mps import split_zgemm
    rng = np.random.default_rng(m + k)
    A = rng.standard_normal((k, m)) + 1j * rng.standard_normal((k, m))
    A *= (2.0 ** rng.integers(-20, 20, size=m))[None, :]
    Ah = np.ascontiguousarray(A.conj().T)
    C = split_zgemm(torch.from_numpy(Ah).cuda(), torch.from_numpy(A).cuda(), 8).cpu().numpy()
    assert np.array_equal(C, C.conj().T)
    assert np.all(np.diag(C).imag == 0)
    bound = np.abs(Ah) @ np.abs(A)
    assert np.max(np.abs(C - Ah @ A) / bound) < 8e-15


# ------------------------------------------------------------- split updates ---

def split_mps(n, chi_max, cutoff):
    from paper_1111_3124_gb300.mps import MPS, PREC_SPLIT
    return MPS(n, chi_max, cutoff, PREC_SPLIT)


def test_split_n10_brickwork_all_amplitudes(torch):
    c = C.WORKLOADS[C.N10]
    n = c["n"]
    layers = C.workload_circuit(C.N10)
    g = split_mps(n, c["chi_max"], c["cutoff"])
    g.run_layers(layers)
    ref = oracle_run(n, layers, c["chi_max"], c["cutoff"])
    sv = StateVector(n)
    for layer in layers:
        for site, U in layer:
            sv.apply(list(range(site, site + {2: 1, 4: 2, 8: 3}[U.shape[0]])), U)
    a = g.amplitudes(all_bits(n))
    assert np.max(np.abs(a - sv.vector())) < 1e-10
    for b in range(n - 1):
        assert spectrum_err(g.schmidt(b), ref.schmidt(b)) < 1e-12


def test_split_truncating_circuit_vs_oracle(torch):
    n, chi_max, cutoff = 12, 8, 1e-12
    layers = C.brickwork(n, 8, np.random.default_rng(55))
    g = split_mps(n, chi_max, cutoff)
    g.run_layers(layers)
    ref = oracle_run(n, layers, chi_max, cutoff)
    for b in range(n - 1):
        assert spectrum_err(g.schmidt(b), ref.schmidt(b)) < 1e-12
    bits = np.random.default_rng(1).integers(0, 2, size=(64, n)).astype(np.uint8)
    assert np.max(np.abs(g.amplitudes(bits) - np.array([ref.amplitude(b) for b in bits]))) < 1e-10


@pytest.mark.parametrize("chi,chi_max", [((1, 3, 5, 2, 1), 64), ((1, 37, 45, 29, 1), 64),
                                         ((1, 70, 97, 50, 1), 128), ((1, 40, 40, 40, 1), 48),
                                         ((1, 256, 256, 256, 1), 256)])
def test_split_single_update_vs_oracle(torch, chi, chi_max):
    n = len(chi) - 1
    state = random_state(n, chi, sum(chi))
    U = C.haar_unitary(4, np.random.default_rng(sum(chi) + 1))
    ref = oracle.OracleMPS(n, chi_max, 1e-12)
    ref.set_state(*state)
    ref.apply_gate(1, U)
    g = split_mps(n, chi_max, 1e-12)
    g.import_state(*state)
    g.apply_gate(1, U)
    _, rg, rl = ref.get_state()
    _, gg, gl = g.export()
    assert len(gl[1]) == len(rl[1])
    assert spectrum_err(gl[1], rl[1]) < 1e-12
    tg, tr = two_site_tensor(gg, gl, 1), two_site_tensor(rg, rl, 1)
    assert np.max(np.abs(tg - tr)) < 1e-11 * np.max(np.abs(tr))


# ------------------------------------------------ three-site (U(8)) updates ---

@pytest.mark.parametrize("chi,chi_max", [((1, 9, 13, 11, 7, 1), 128), ((1, 33, 40, 21, 17, 1), 128),
                                         ((1, 20, 20, 20, 20, 1), 24), ((1, 128, 128, 128, 128, 1), 128)])
def test_split_three_site_update_vs_oracle(torch, chi, chi_max):
    """U(8) on sites 1..3 of a 5-site random state in split mode: both splits
    run the split SVD (the second one's working matrix moved from T to A and
    back). The third case truncates both splits to chi_max; the last has the
    three-site workload's chi = 128 shape (theta 256 x 512)."""
    from tests.helpers import three_site_tensor
    n = len(chi) - 1
    state = random_state(n, chi, 7 * sum(chi))
    U = C.haar_unitary(8, np.random.default_rng(7 * sum(chi) + 1))
    ref = oracle.OracleMPS(n, chi_max, 1e-12)
    ref.set_state(*state)
    ref.apply_gate(1, U)
    g = split_mps(n, chi_max, 1e-12)
    g.import_state(*state)
    g.apply_gate(1, U)
    _, rg, rl = ref.get_state()
    _, gg, gl = g.export()
    for b in (1, 2):
        assert len(gl[b]) == len(rl[b])
        assert spectrum_err(gl[b], rl[b]) < 1e-12
    tg, tr = three_site_tensor(gg, gl, 1), three_site_tensor(rg, rl, 1)
    assert np.max(np.abs(tg - tr)) < 1e-11 * np.max(np.abs(tr))


@pytest.mark.parametrize("seed", [0, 1])
def test_split_mixed_1_2_3_site_gates_vs_statevector(torch, seed):
    from tests.test_oracle import random_layers
    rng = np.random.default_rng(300 + seed)
    n = 8
    layers = random_layers(n, 6, rng)
    g = split_mps(n, 64, 0.0)
    for layer in layers:
        for site, U in layer:
            g.apply_gate(site, U)
    sv = StateVector(n)
    for layer in layers:
        for site, U in layer:
            sv.apply(list(range(site, site + {2: 1, 4: 2, 8: 3}[U.shape[0]])), U)
    np.testing.assert_allclose(g.amplitudes(all_bits(n)), sv.vector(), atol=1e-10)


def test_split_ghz_prefix_and_u8_layers_vs_oracle(torch):
    """GHZ ladder then two shifted-brick layers of U(8), n = 12, chi_max 32:
    Schmidt values {1/sqrt 2, 1/sqrt 2} after the prefix, oracle parity after
    the U(8) layers."""
    n = 12
    layers = C.ghz_prefix(n) + C.u8_shifted_brick(n, 2, np.random.default_rng(91))
    g = split_mps(n, 32, 1e-12)
    prefix = len(C.ghz_prefix(n))
    g.run_layers(layers[:prefix])
    for b in range(n - 1):
        np.testing.assert_allclose(g.schmidt(b), [2 ** -0.5, 2 ** -0.5], atol=1e-14)
    g.run_layers(layers[prefix:])
    ref = oracle_run(n, layers, 32, 1e-12)
    for b in range(n - 1):
        assert spectrum_err(g.schmidt(b), ref.schmidt(b)) < 1e-12
    bits = np.random.default_rng(5).integers(0, 2, size=(64, n)).astype(np.uint8)
    assert np.max(np.abs(g.amplitudes(bits) - np.array([ref.amplitude(b) for b in bits]))) < 1e-10
