"""bench.py on the CPU: the multi-rank timing reduction over two gloo ranks
(max over ranks, whole-job throughput = units of all ranks / slowest time),
and the reference arm (the oracle on the host cores): its JSON line on rank 0
and no output from the other ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_rank_reduction_two_gloo_ranks():
    pytest.importorskip("torch")
    port, world = _free_port(), 2
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, os.path.join(ROOT, "tests", "multirank_worker.py")],
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["t_step"] == 2.0 and o["t_e2e"] == 20.0  # the slowest rank of each quantity
        assert o["value"] == pytest.approx(630 * 2 / 2.0)


def test_reduce_max_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.job_throughput(630, 1, 2.0) == 315.0


def _run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "1"], env=env, capture_output=True, text=True,
                          timeout=600, cwd=ROOT)


def test_reference_arm_line():
    r = _run_reference({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "updates/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"] == "n64_d20_u4_rz_chi256"


def test_reference_arm_other_ranks_exit_without_work():
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_nominal_work_count():
    """Nominal binary64 work per two-site update: 32 chi^3 (theta) + 704 chi^3
    (Golub-Reinsch SVD of the complex 2chi x 2chi theta) at square chi; the
    wide case is counted on its transpose; the pass reads the bonds around
    each gate (1 at the chain's ends) and skips single-site layers."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    assert bench.nominal_update_flops(256, 256, 256) == (32 * 256 ** 3, 704 * 256 ** 3)
    assert bench.nominal_update_flops(4, 8, 16) == bench.nominal_update_flops(16, 8, 4)
    m_, n_ = 32, 8  # chi_l = 16, chi_r = 4
    assert bench.nominal_update_flops(16, 8, 4) == (8 * m_ * n_ * 8, 4 * (14 * m_ * n_ ** 2 + 8 * n_ ** 3))

    class Stub:  # bond dimensions 2, 3, 5 of a 4-site chain; records the calls
        def __init__(self):
            self.calls = []

        def reset(self):
            self.calls.append("reset")

        def bond_dims(self):
            return np.array([2, 3, 5], dtype=np.int32)

        def apply_layer_device(self, s, dU, k):
            self.calls.append((k, tuple(s.tolist())))

        def sync(self):
            self.calls.append("sync")

    layers = [(2, np.array([0, 2], dtype=np.int32), None), (1, np.array([0, 1, 2, 3], dtype=np.int32), None),
              (2, np.array([1], dtype=np.int32), None)]
    stub = Stub()
    got = bench.step_nominal_flops(stub, layers, 4)
    parts = [bench.nominal_update_flops(1, 2, 3), bench.nominal_update_flops(3, 5, 1),
             bench.nominal_update_flops(2, 3, 5)]
    assert got["theta"] == sum(t for t, _ in parts) and got["svd"] == sum(v for _, v in parts)
    assert got["total"] == got["theta"] + got["svd"]
    assert stub.calls == ["reset", (2, (0, 2)), (1, (0, 1, 2, 3)), (2, (1,)), "sync"]


def test_fp32_launch_mode_lookup():
    """The roofline names the fp32 sweep kernel and picks its captured traffic
    from the tuning table as the library applies it: the first entry whose
    nw_max covers the width, else the last; no table means the library's
    default (block width 16, scheduled launch of 256-thread CTAs)."""
    sys.path.insert(0, ROOT)
    import bench
    table = [(64, 16, 2), (128, 8, 0), (256, 16, 3), (512, 16, 1)]
    assert bench.f32_mode(table, 40) == (16, 2)
    assert bench.f32_mode(table, 128) == (8, 0)
    assert bench.f32_mode(table, 200) == (16, 3)
    assert bench.f32_mode(table, 4096) == (16, 1)  # beyond the last entry: the last entry
    assert bench.f32_mode(None, 512) == (16, 2) and bench.f32_mode([], 512) == (16, 2)
    assert "k_jacobi_f32_sched<16, 256>" in bench.f32_kernel_name(None, 512)
    assert "k_jacobi_f32_sched<16, 384>" in bench.f32_kernel_name(table, 200)
    assert "k_rot_tc" in bench.f32_kernel_name(table, 512)
    assert "k_jacobi_pair_f32<8>" in bench.f32_kernel_name(table, 100)
    assert 2 in bench.F32_CAPTURED and 0 in bench.F32_CAPTURED
