"""The no-allocation two-site update (mps_gate2_update_noalloc) against the
handle-based update (mps_apply_gate), called through the C ABI on the GPU.

Collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test. It must pass alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest

from paper_1111_3124_gb300 import circuits as C
from tests.helpers import spectrum_err, two_site_tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1111_3124_gb300 import build as B
    B.build()
    return torch


def _device_tensors(torch, state, cap):
    gammas, lams = state
    def gam(g):
        out = np.zeros((2, cap, cap), dtype=np.complex128)
        out[:, :g.shape[1], :g.shape[2]] = g
        return torch.from_numpy(out).cuda()
    def lam(v):
        out = np.zeros(cap)
        out[:len(v)] = v
        return torch.from_numpy(out).cuda()
    chi = torch.tensor([gammas[1].shape[1], gammas[1].shape[2], gammas[2].shape[2]], dtype=torch.int32).cuda()
    return gam(gammas[1]), gam(gammas[2]), lam(lams[0]), lam(lams[1]), lam(lams[2]), chi


def test_noalloc_matches_apply_gate_two_calls(torch_cuda):
    torch = torch_cuda
    from paper_1111_3124_gb300.mps import MPS, gate2_update_noalloc
    cap, cutoff = 32, 1e-12
    chi = (1, 21, 30, 29, 13, 1)   # ragged; theta is 42 x 58 and both updates truncate to chi_max = 32
    rng = np.random.default_rng(4242)
    state = C.random_vidal_state(5, chi, rng)
    U1, U2 = C.haar_unitary(4, rng), C.haar_unitary(4, rng)

    ref = MPS(5, cap, cutoff)
    ref.import_state(*state)
    gl, gr, ll, lm, lr, dchi = _device_tensors(torch, state, cap)
    for U in (U1, U2):   # two calls in a row, the second on the first's output
        ref.apply_gate(1, U)
        gate2_update_noalloc(gl, gr, ll, lm, lr, dchi, cap, cutoff, U)
        torch.cuda.synchronize()
        _, rg, rlam = ref.export()
        k = int(dchi[1].item())
        assert k == len(rlam[1])
        assert int(dchi[0].item()) == chi[1] and int(dchi[2].item()) == chi[3]
        g_l = gl.cpu().numpy()[:, :chi[1], :k]
        g_r = gr.cpu().numpy()[:, :k, :chi[3]]
        lam_m = lm.cpu().numpy()[:k]
        assert spectrum_err(lam_m, rlam[1]) < 1e-12
        mine = two_site_tensor([rg[0], g_l, g_r, rg[3], rg[4]], [rlam[0], lam_m, rlam[2], rlam[3]], 1)
        theirs = two_site_tensor(rg, rlam, 1)
        assert np.max(np.abs(mine - theirs)) < 1e-11 * np.max(np.abs(theirs))


def test_noalloc_at_its_size_limit_matches_the_oracle(torch_cuda):
    """chi_max = 64 with every touched bond saturated (theta 128 x 128, the
    largest the fixed scratch array holds), two calls in a row, checked
    against the CPU oracle and against mps_apply_gate."""
    torch = torch_cuda
    import oracle
    from paper_1111_3124_gb300.mps import MPS, gate2_update_noalloc
    cap, cutoff = 64, 1e-12
    chi = (1, 64, 64, 64, 64, 1)
    rng = np.random.default_rng(6464)
    state = C.random_vidal_state(5, chi, rng, decay=2.0)
    U1, U2 = C.haar_unitary(4, rng), C.haar_unitary(4, rng)
    ref = MPS(5, cap, cutoff)
    ref.import_state(*state)
    orc = oracle.OracleMPS(5, cap, cutoff)
    orc.set_state(*state)
    gl, gr, ll, lm, lr, dchi = _device_tensors(torch, state, cap)
    for U in (U1, U2):
        ref.apply_gate(1, U)
        orc.apply_gate(1, U)
        gate2_update_noalloc(gl, gr, ll, lm, lr, dchi, cap, cutoff, U)
        torch.cuda.synchronize()
        k = int(dchi[1].item())
        _, og, olam = orc.get_state()
        assert k == len(olam[1]) == 64
        _, rg, rlam = ref.export()
        g_l = gl.cpu().numpy()[:, :64, :k]
        g_r = gr.cpu().numpy()[:, :k, :64]
        lam_m = lm.cpu().numpy()[:k]
        assert spectrum_err(lam_m, olam[1]) < 1e-12
        assert spectrum_err(lam_m, rlam[1]) < 1e-12
        mine = two_site_tensor([og[0], g_l, g_r, og[3], og[4]], [olam[0], lam_m, olam[2], olam[3]], 1)
        theirs = two_site_tensor(og, olam, 1)
        assert np.max(np.abs(mine - theirs)) < 1e-11 * np.max(np.abs(theirs))
        # continue both GPU paths from the oracle's state so the second call is teacher-forced
        ref.import_state(og, olam)
        st = _device_tensors(torch, (og, olam), cap)
        for dst, src in zip((gl, gr, ll, lm, lr, dchi), st):
            dst.copy_(src)


def test_noalloc_rejects_oversized_chi_max(torch_cuda):
    torch = torch_cuda
    from paper_1111_3124_gb300.mps import MPSError, MPS_ERR_TOO_LARGE, gate2_update_noalloc
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    chi = torch.ones(3, dtype=torch.int32, device="cuda")
    with pytest.raises(MPSError) as e:
        gate2_update_noalloc(z, z, z, z, z, chi, 65, 0.0, np.eye(4))
    assert e.value.code == MPS_ERR_TOO_LARGE


def test_noalloc_rejects_bond_dims_beyond_chi_max(torch_cuda):
    torch = torch_cuda
    from paper_1111_3124_gb300.mps import MPSError, MPS_ERR_ARG, gate2_update_noalloc
    z = torch.zeros(2 * 16 * 16, dtype=torch.complex128, device="cuda")
    lam = torch.ones(16, dtype=torch.float64, device="cuda")
    chi = torch.tensor([1, 17, 1], dtype=torch.int32, device="cuda")
    with pytest.raises(MPSError) as e:
        gate2_update_noalloc(z, z, lam, lam, lam, chi, 16, 0.0, np.eye(4))
    assert e.value.code == MPS_ERR_ARG
