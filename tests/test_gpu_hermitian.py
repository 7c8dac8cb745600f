"""The Hermitian-matrix workload on the GPU (mps_heev_batched,
mps_hermitian_function_batched, mps_fid_batched, mps_dft_abs_batched) against
the oracle (numpy eigh, scipy expm, the definition of the record, numpy FFT)
and the closed forms of the paper's two-spin NMR example (Sec. 2.1).

Tolerances: a backward-stable Hermitian eigensolver gives eigenvalues to
O(D eps ||H||) absolute; products of D x D unitaries add O(D eps) relative;
the record's phases (lambda_j - lambda_k) t reach 6e4 rad at the example's
last sample, where one ulp of the phase is ~1e-11."""
import numpy as np
import pytest

from oracle import hermitian as O
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("D", [1, 2, 3, 8, 17, 32, 64])
def test_heev_random_batch_vs_eigh(D):
    from paper_1111_3124_gb300.mps import heev
    H = C.random_hermitian(48, D, np.random.default_rng(100 + D))
    w, V = heev(_dev(H))
    w, V = w.cpu().numpy(), V.cpu().numpy()
    for b in range(H.shape[0]):
        wr, _ = O.heev(H[b])
        nrm = np.linalg.norm(H[b])
        assert np.max(np.abs(w[b] - wr)) < 8 * D * 1.1e-16 * nrm
        assert np.max(np.abs(V[b].conj().T @ V[b] - np.eye(D))) < 8 * D * 1.1e-16
        assert np.max(np.abs(V[b] @ np.diag(w[b]) @ V[b].conj().T - H[b])) < 8 * D * 1.1e-16 * nrm


def test_heev_degenerate_spectra():
    from paper_1111_3124_gb300.mps import heev, hermitian_last_stats
    heis = np.kron(C.X, C.X) + np.kron(C.Y, C.Y) + np.kron(C.Z, C.Z)
    H3 = C.spin_hamiltonians(1, 3, np.random.default_rng(1), shift_hz=0.0, j_hz=1.0)[0]  # no offsets: degenerate
    for H in (heis, H3, np.zeros((4, 4), dtype=np.complex128), np.eye(8, dtype=np.complex128)):
        w, V = heev(_dev(H[None]))
        w, V = w.cpu().numpy()[0], V.cpu().numpy()[0]
        assert np.allclose(w, O.heev(H)[0], atol=1e-13)
        assert np.allclose(V @ np.diag(w) @ V.conj().T, H, atol=1e-13)
        assert np.allclose(V.conj().T @ V, np.eye(len(w)), atol=1e-13)
    assert hermitian_last_stats()["max_sweeps"] >= 1


def test_exp_and_thermal_vs_oracle():
    from paper_1111_3124_gb300.mps import expm_hermitian, thermal_state
    H = C.spin_hamiltonians(16, 4, np.random.default_rng(2))
    Hd = _dev(H)
    for a in (-1j * 1e-3, -2.0e-3, 0.5e-3 - 1e-3j):
        E = expm_hermitian(2 * np.pi * Hd, a).cpu().numpy()
        for b in range(H.shape[0]):
            ref = O.expm(2 * np.pi * H[b], a)
            assert np.max(np.abs(E[b] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))
    beta = 1e-3
    R = thermal_state(Hd, beta).cpu().numpy()
    for b in range(H.shape[0]):
        ref = O.thermal(H[b], beta)
        assert np.max(np.abs(R[b] - ref)) < 1e-13
        assert abs(np.trace(R[b]) - 1) < 1e-14


def test_two_spin_example_thermal_fid_and_spectrum():
    """Sec. 2.1 end to end: rho = exp_H(-beta H) / Tr, Y_90 pulse, <X_1> every
    dt for N = 32768 samples, zero padding to 2N, |DFT|: the record equals its
    closed form and the two strongest lines sit at 2 w1 +- 2 J12."""
    from paper_1111_3124_gb300.mps import dft_abs, fid, thermal_state
    ex = C.nmr_example()
    rho = thermal_state(_dev(ex["H"][None]), ex["beta"])
    rho_h = rho.cpu().numpy()[0]
    assert np.max(np.abs(rho_h - O.thermal(ex["H"], ex["beta"]))) < 1e-16
    s = fid(rho, _dev((2 * np.pi * ex["H"])[None]), _dev(ex["O"][None]), ex["dt"], ex["N"], P=_dev(ex["P"][None]))
    s = s.cpu().numpy()[0]
    from tests.test_oracle_hermitian import _fid_closed_form
    ref = _fid_closed_form(ex, np.arange(ex["N"]))
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(s.real - ref)) < 1e-9 * scale
    assert np.max(np.abs(s.imag)) < 1e-9 * scale
    ms = [0, 5, 4096, 32767]
    so = O.fid(O.thermal(ex["H"], ex["beta"]), 2 * np.pi * ex["H"], ex["O"], ex["dt"], ms, P=ex["P"])
    assert np.max(np.abs(s[ms] - so)) < 1e-9 * scale
    n_out = 2 * ex["N"]
    spec = dft_abs(_dev(s[None]), n_out).cpu().numpy()[0]
    assert np.max(np.abs(spec - O.dft_abs(s, n_out))) < 1e-9 * np.max(spec)
    df = 1.0 / (n_out * ex["dt"])
    half = spec[: n_out // 2]
    top = sorted(np.argsort(half)[-2:])
    want = sorted(round((2 * ex["w1"] + 2 * ex["J"] * z) / df) for z in (-1, 1))
    assert all(abs(a - b) <= 1 for a, b in zip(top, want)), (top, want)


def test_fid_batch_vs_oracle_and_dft_vs_fft():
    from paper_1111_3124_gb300.mps import dft_abs, fid, thermal_state
    spins = 3
    H = C.spin_hamiltonians(8, spins, np.random.default_rng(3))
    P = C.kron_all(*[C.Y90] * spins)
    Ox = sum(C.kron_all(*[C.X if q == k else C.I2 for q in range(spins)]) for k in range(spins))
    Hd = _dev(2 * np.pi * H)
    rho = thermal_state(_dev(H), 1e-2)
    dt, N = 2.5e-4, 1000
    s = fid(rho, Hd, _dev(np.broadcast_to(Ox, H.shape).copy()), dt, N, P=_dev(np.broadcast_to(P, H.shape).copy()))
    s = s.cpu().numpy()
    rho_h = rho.cpu().numpy()
    ms = [0, 1, 333, 999]
    for b in range(H.shape[0]):
        ref = O.fid(rho_h[b], 2 * np.pi * H[b], Ox, dt, ms, P=P)
        assert np.max(np.abs(s[b, ms] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))
    spec = dft_abs(_dev(s), 4096).cpu().numpy()
    for b in range(H.shape[0]):
        ref = O.dft_abs(s[b], 4096)
        assert np.max(np.abs(spec[b] - ref)) < 1e-11 * np.max(ref)


def test_argument_checks():
    import torch
    from paper_1111_3124_gb300.mps import MPSError, MPS_ERR_ARG, MPS_ERR_TOO_LARGE, dft_abs, heev
    with pytest.raises(MPSError) as e:
        heev(torch.zeros((1, 65, 65), dtype=torch.complex128, device="cuda"))
    assert e.value.code == MPS_ERR_TOO_LARGE
    with pytest.raises(MPSError) as e:
        dft_abs(torch.zeros((1, 10), dtype=torch.complex128, device="cuda"), 12)
    assert e.value.code == MPS_ERR_ARG


def test_thermal_deviation_at_300K_and_its_record():
    """At 300 K with Hz-scale couplings the thermal state differs from I/D in
    the 10th digit; its deviation (kind 2, expm1 weights) keeps full relative
    accuracy, and so does the record of a traceless observable built on it."""
    from paper_1111_3124_gb300.mps import fid, thermal_deviation
    spins = 4
    H = C.spin_hamiltonians(16, spins, np.random.default_rng(12))
    beta = C.PLANCK / C.BOLTZMANN / 300.0
    dev = thermal_deviation(_dev(H), beta)
    dev_h = dev.cpu().numpy()
    P = C.kron_all(*[C.Y90] * spins)
    Ox = sum(C.kron_all(*[C.X if q == k else C.I2 for q in range(spins)]) for k in range(spins))
    dt, N = 2.5e-4, 512
    s = fid(dev, _dev(2 * np.pi * H), _dev(np.broadcast_to(Ox, H.shape).copy()), dt, N,
            P=_dev(np.broadcast_to(P, H.shape).copy())).cpu().numpy()
    ms = [0, 7, 511]
    for b in range(H.shape[0]):
        ref = O.thermal_deviation(H[b], beta)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(dev_h[b] - ref)) < 1e-12 * scale
        fr = O.fid(ref, 2 * np.pi * H[b], Ox, dt, ms, P=P)
        assert np.max(np.abs(s[b, ms] - fr)) < 1e-11 * np.max(np.abs(fr))
