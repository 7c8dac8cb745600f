#!/usr/bin/env python
"""Benchmark: two-site gate updates per second on the n=64, depth-20
Haar-random U(4) brickwork (+ RZ phases) workload at chi_max = 256.

One step = the whole circuit from |0...0> (630 two-site updates: theta
formation, Jacobi SVD, truncation, rewrite), inputs resident in HBM.
Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--prec split|fp64] [--no-fp64-compare]
  python bench.py --profile-layer [--n 64] [--chi 256] [--layers 1] [--prec split|fp64]

--profile-layer runs the case that hardware-counter captures use: brickwork
layers of Haar U(4) updates on a synthetic Vidal state with every bond at
min(chi, 2^b, 2^(n-b)), so that every update works on a saturated 2chi x 2chi
theta after only a few setup launches. It prints a one-line summary, not the
bench line.

The headline is the split-precision path (bf16-sliced tensor-core products,
fp32 preconditioning sweeps, binary64 angles, tests and polish); the native
binary64 path is timed beside it on the same workload (`fp64_path`), with the
split result's deviation from it.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "two-site gate updates/s at χ=256, mixed-prec vs FP64 on GB300, amp err ≤10^-10".replace(
    "10^-10", "1e-10")
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
KERNEL_CLASSES = ["jacobi_f64", "theta_contract_f64", "truncate_rewrite", "split_gemm_tc", "jacobi_f32", "split_aux"]


def measure_alu_peaks():
    """fp32 and binary64 throughput of the library GEMM (torch.matmul on the
    CUDA cores, tf32 off), best of three at 8192^3 / 4096^3: the measured ALU
    peaks the Jacobi kernels are held against."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    out = {}
    for name, dt, n in (("fp32", torch.float32, 8192), ("fp64", torch.float64, 4096)):
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        torch.matmul(a, b)
        best = float("inf")
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[name + "_tflops"] = 2.0 * n ** 3 / best / 1e12
        del a, b
    out["how"] = "torch.matmul fp32 8192^3 and fp64 4096^3 (tf32 off), best of 3, CUDA events"
    return out


def peaks():
    """Roofline denominators. Tensor: MEASURED_PEAKS.json (bf16, sustained for a
    kernel timed inside a long step). ALU: GB300 unit counts x max SM clock
    (152 SMs, 2070 MHz; binary64 2 FMA/clk/SM, fp32 128 FMA/clk/SM)."""
    try:
        mp = json.load(open(PEAKS))
    except (OSError, ValueError):
        mp = {}
    sm_mhz = float(mp.get("sm_max_mhz", 2070.0))
    return {
        "bf16_tflops": float(mp.get("bf16_tflops_sustained", 1700.0)),
        "bf16_source": "MEASURED_PEAKS.json bf16_tflops_sustained" if "bf16_tflops_sustained" in mp else "fallback",
        "fp64_tflops": 152 * 2 * 2 * sm_mhz * 1e6 / 1e12,
        "fp32_tflops": 152 * 128 * 2 * sm_mhz * 1e6 / 1e12,
        "sm_mhz": sm_mhz,
    }


def args_parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--prec", default="split", choices=["fp64", "split"])
    p.add_argument("--no-fp64-compare", action="store_true",
                   help="skip timing the native binary64 path beside the split path")
    p.add_argument("--cpu-sample", type=int, default=2, help="oracle updates timed for cpu_baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--n", type=int, default=None, help="override the qubit count (small profiling cases)")
    p.add_argument("--depth", type=int, default=None, help="override the circuit depth")
    p.add_argument("--profile-layer", action="store_true", help="run the saturated-layer capture case")
    p.add_argument("--path", default="program", choices=["program", "eager"],
                   help="timed path: the circuit recorded once and replayed as a CUDA graph, or host-driven passes")
    p.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the binary64 comparison")
    p.add_argument("--no-extra-configs", action="store_true", help="skip the three-site and many-circuit lines")
    p.add_argument("--batch-circuits", type=int, default=32, help="circuits of the many-circuit line")
    p.add_argument("--retune", action="store_true", help="ignore the tuner's cache")
    p.add_argument("--chi", type=int, default=256, help="bond dimension of the saturated-layer case")
    p.add_argument("--layers", type=int, default=1, help="layers of the saturated-layer case")
    p.add_argument("--profile-dd", action="store_true",
                   help="run the double-word capture case (2 circuits, n=32, chi_max=32, 8 layers)")
    p.add_argument("--profile-hermitian", action="store_true",
                   help="run the Hermitian-workload capture case (1024 five-spin systems)")
    return p.parse_args()


ARGS = None


def workload():
    from paper_1111_3124_gb300 import circuits as C
    c = dict(C.WORKLOADS[C.N64_CHI256])
    n = ARGS.n if ARGS and ARGS.n else c["n"]
    depth = ARGS.depth if ARGS and ARGS.depth else c["depth"]
    if (n, depth) != (c["n"], c["depth"]):
        c["name"] = "n%d_d%d_u4_rz_chi%d" % (n, depth, c["chi_max"])
    c["n"], c["depth"] = n, depth
    layers = C.workload_circuit(C.N64_CHI256, n=n, depth=depth)
    return c, layers, C.count_updates(layers)


def grouped(layers):
    """Each layer -> list of (k, sites, Us) with same-size gates batched."""
    out = []
    for layer in layers:
        by_k = {}
        for site, U in layer:
            by_k.setdefault(U.shape[0], []).append((site, U))
        for d in sorted(by_k):
            k = {2: 1, 4: 2, 8: 3}[d]
            gs = by_k[d]
            out.append((k, np.array([s for s, _ in gs], dtype=np.int32),
                        np.ascontiguousarray(np.stack([U for _, U in gs]).astype(np.complex128))))
    return out


# ----------------------------------------------------------------- clocks ---

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------ CPU oracle ---

def oracle_sample(n_updates: int):
    """The oracle (as it stands, one host thread) on a bounded sample of the
    workload: steady-state two-site updates at chi_L = chi = chi_R = 256
    (theta 512 x 512, truncated to 256) on a synthetic saturated state."""
    import oracle
    from paper_1111_3124_gb300 import circuits as C
    t_total = 0.0
    for i in range(n_updates):
        rng = np.random.default_rng(9000 + i)
        state = C.random_vidal_state(4, (1, 256, 256, 256, 1), rng, decay=2.0)
        m = oracle.OracleMPS(4, 256, 1e-12)
        m.set_state(*state)
        U = C.haar_unitary(4, rng)
        t0 = time.perf_counter()
        m.apply_gate(1, U)
        t_total += time.perf_counter() - t0
    return n_updates / t_total, t_total


def cpu_baseline_obj(n_updates: int):
    v, t = oracle_sample(n_updates)
    return {"value": v, "unit": "updates/s", "cores": 1, "kind": "oracle",
            "sample": "%d steady-state two-site updates at chi=256 (theta 512x512 -> 256) on a synthetic "
                      "saturated Vidal state, binary64 oracle, one host thread, %.1f s" % (n_updates, t)}


# --------------------------------------------------------------- ref arm ---

def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c, layers, nup = workload()
    for _ in range(a.warmup):
        oracle_sample(1)
    times = []
    for _ in range(a.steps):
        _, t = oracle_sample(1)
        times.append(t)
    v = len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "updates/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": c["name"], "n": c["n"], "depth": c["depth"],
                                            "chi_max": c["chi_max"], "cutoff": c["cutoff"],
                                            "step": "one steady-state update (bounded sample)"},
            "cpu_baseline": {"value": v, "unit": "updates/s", "cores": 1, "kind": "oracle",
                             "sample": "one chi=256 update per step on a synthetic saturated state"},
            "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------- nominal work ---

def nominal_update_flops(chi_l: int, chi_m: int, chi_r: int):
    """Nominal binary64 work of one two-site update on bonds (chi_l, chi_m,
    chi_r): (theta, svd) with theta as a complex GEMM, 8 flops per
    multiply-add over (2 chi_l) x (2 chi_r) x chi_m, and the SVD of the
    complex M x N theta by the Golub-Reinsch count 4 (14 M N^2 + 8 N^3),
    M >= N. At chi = 256 everywhere: 32 chi^3 + 704 chi^3 = 12.4 GFLOP."""
    m, n = 2 * chi_l, 2 * chi_r
    if m < n:
        m, n = n, m
    return 8.0 * m * n * chi_m, 4.0 * (14.0 * m * n * n + 8.0 * n ** 3)


def step_nominal_flops(m, dev_layers, n: int) -> dict:
    """One untimed pass of the circuit, summing the nominal work of every
    two-site update from the bond dimensions before its layer."""
    theta = svd = 0.0
    m.reset()
    for k, s, dU in dev_layers:
        if k == 2:
            bd = m.bond_dims()
            for site in s.tolist():
                chi_l = int(bd[site - 1]) if site > 0 else 1
                chi_r = int(bd[site + 1]) if site + 1 < n - 1 else 1
                t, v = nominal_update_flops(chi_l, int(bd[site]), chi_r)
                theta += t
                svd += v
        m.apply_layer_device(s, dU, k)
    m.sync()
    return {"total": theta + svd, "theta": theta, "svd": svd}


# ------------------------------------------------------------ multi-rank ---

def reduce_max(values, world: int):
    """Max over the ranks of each value: the slowest rank sets the job time.
    One rank: the values unchanged. NCCL reduces on the device, gloo on the host."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / seconds


# ------------------------------------------------------------- GPU arm ---

def program_passes(dev_layers):
    """The circuit's device layers as recorded-program passes (one handle)."""
    return [(k, [(0, int(q)) for q in s], dU) for k, s, dU in dev_layers]


def oracle_check(prec, n_updates: int):
    """The saturated chi = 256 update of the CPU-baseline sample (synthetic
    saturated state, Haar U(4), theta 512 x 512 cut to 256) on the GPU, against
    the oracle: largest Schmidt-value error relative to lambda_0 and largest
    error of the reconstructed two-site tensor relative to its largest entry."""
    import oracle
    from paper_1111_3124_gb300 import circuits as C
    from paper_1111_3124_gb300.mps import MPS
    spec, theta = 0.0, 0.0
    for i in range(n_updates):
        rng = np.random.default_rng(9000 + i)
        state = C.random_vidal_state(4, (1, 256, 256, 256, 1), rng, decay=2.0)
        U = C.haar_unitary(4, rng)
        orc = oracle.OracleMPS(4, 256, 1e-12)
        orc.set_state(*state)
        orc.apply_gate(1, U)
        g = MPS(4, 256, 1e-12, prec)
        g.import_state(*state)
        g.apply_gate(1, U)
        _, og, ol = orc.get_state()
        _, gg, gl = g.export()
        g.close()
        if len(ol[1]) != len(gl[1]):
            return {"max_spectrum_err": float("inf"), "max_theta_err": float("inf"), "updates": n_updates}
        spec = max(spec, float(np.max(np.abs(ol[1] - gl[1])) / ol[1][0]))
        t_o = np.einsum("a,iac,c,jcb,b->iajb", ol[0], og[1], ol[1], og[2], ol[2])
        t_g = np.einsum("a,iac,c,jcb,b->iajb", gl[0], gg[1], gl[1], gg[2], gl[2])
        theta = max(theta, float(np.max(np.abs(t_o - t_g)) / np.max(np.abs(t_o))))
    return {"max_spectrum_err": spec, "max_theta_err": theta, "updates": n_updates,
            "case": "teacher-forced chi=256 updates of the CPU-baseline sample, GPU vs oracle"}


def run_three_site(prec, steps: int, tune_table=()):
    """Three-site workload: GHZ prefix, then a depth-12 shifted brick of Haar
    U(8) gates on n = 48, chi_max = 128, cutoff 1e-12, as one recorded program."""
    import torch
    from paper_1111_3124_gb300 import circuits as C
    from paper_1111_3124_gb300.mps import MPS, Program, circuit_passes
    c = C.WORKLOADS[C.N48_U8]
    layers = C.workload_circuit(C.N48_U8)
    m = MPS(c["n"], c["chi_max"], c["cutoff"], prec)
    m.set_tuning(list(tune_table))
    prog = Program([m], circuit_passes(layers))
    prog.run()
    m.sync()
    ts = []
    for _ in range(steps):
        m.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prog.run()
        m.sync()
        ts.append(time.perf_counter() - t0)
    lam = [m.schmidt(b) for b in range(0, c["n"] - 1, 7)]
    out = {"workload": c["name"], "updates_per_step": prog.updates, "value": prog.updates / (sum(ts) / len(ts)),
           "unit": "updates/s", "steps": steps, "warmup": 1, "prec": "split" if prec else "fp64",
           "timing": "wall clock around mps_program_run + mps_sync"}
    prog.close()
    m.close()
    del lam
    return out


def run_many_circuits(prec, count: int, steps: int, tune_table=()):
    """Many circuits at once: the first `count` circuits of the 512-circuit
    workload (n in [16, 64], depth in [8, 24], chi_max in {32, 64, 128, 256},
    Haar U(4) brickwork), recorded as one program whose passes hold the same
    depth's layer of every circuit."""
    import torch
    from paper_1111_3124_gb300 import circuits as C
    from paper_1111_3124_gb300.mps import MPS, Program
    specs = C.batch_specs(512)[:count]
    circuits = [C.batch_circuit(i, n, d) for i, (n, d, _) in enumerate(specs)]
    states = [MPS(n, chi, 1e-12, prec) for n, _, chi in specs]
    states[0].set_tuning(list(tune_table))  # the program's work runs with the first handle's settings
    passes = []
    for depth in range(max(d for _, d, _ in specs)):
        gates, mats = [], []
        for i, layers in enumerate(circuits):
            if depth < len(layers):
                for site, U in layers[depth]:
                    gates.append((i, site))
                    mats.append(U)
        if gates:
            passes.append((2, gates, torch.from_numpy(np.stack(mats).astype(np.complex128)).cuda()))
    prog = Program(states, passes)
    prog.run()
    states[0].sync()
    ts = []
    for _ in range(steps):
        for st in states:
            st.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prog.run()
        for st in states:
            st.sync()
        ts.append(time.perf_counter() - t0)
    out = {"workload": "first %d of batch512_n16-64_d8-24_chi32-256" % count, "circuits": count,
           "updates_per_step": prog.updates, "value": prog.updates / (sum(ts) / len(ts)), "unit": "updates/s",
           "steps": steps, "warmup": 1, "prec": "split" if prec else "fp64",
           "timing": "wall clock around mps_program_run + mps_sync of every circuit"}
    prog.close()
    for st in states:
        st.close()
    return out


def run_routing(prec, tune_table=()):
    """Gates on non-neighbours (Sec. 3.2's applyU on qubits 0 and 2): distance-2
    Haar U(4) gates on a chi_max = 64 state of 32 qubits, routed as one U(8)
    update each, or as SWAP, gate, SWAP (three two-site updates each)."""
    import torch
    from paper_1111_3124_gb300 import circuits as C
    from paper_1111_3124_gb300.mps import MPS
    n, chi = 32, 64
    rng = np.random.default_rng(C.SEED_BASE + 31)
    base = C.brickwork(n, 6, rng)
    gates = [((4 * j, 4 * j + 2), C.haar_unitary(4, rng)) for j in range(n // 4)]
    gates += [((4 * j + 3, 4 * j + 1), C.haar_unitary(4, rng)) for j in range(n // 4)]
    out, amps = {}, {}
    bits = np.random.default_rng(7).integers(0, 2, size=(64, n)).astype(np.uint8)
    for route in ("embed", "swap"):
        m = MPS(n, chi, 1e-12, prec)
        m.set_tuning(list(tune_table))
        m.run_layers(base)
        m.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for (q, U) in gates:
            m.apply_gate_on(list(q), U, route=route)
        m.sync()
        dt = time.perf_counter() - t0
        amps[route] = m.amplitudes(bits)
        out[route] = {"seconds": dt, "gates": len(gates), "gates_per_s": len(gates) / dt,
                      "updates": len(gates) * (1 if route == "embed" else 3),
                      "update_kind": "three-site" if route == "embed" else "two-site"}
        m.close()
    out["max_amp_diff_between_routes"] = float(np.max(np.abs(amps["embed"] - amps["swap"])))
    out["workload"] = "n=32, chi_max=64 after 6 brickwork layers; 16 distance-2 Haar U(4) gates"
    return out


def run_dd(fp64_peak_tflops: float, circuits: int = 8, steps: int = 2, depth: int = 20):
    """Beyond binary64: `circuits` independent n = 32, depth-20 circuits of
    Haar U(4) gates with RZ phases (gates unitary to ~1e-32, given as hi + lo),
    chi_max = 32, cutoff 1e-28, each on its own double-word handle and CUDA
    stream, gates resident on the device; plus the error against the oracle
    in binary128 on an n = 8 circuit of the same kind."""
    import torch
    import oracle
    from paper_1111_3124_gb300 import circuits as C
    from paper_1111_3124_gb300.mps import MPSDD
    n, chi, cutoff = 32, 32, 1e-28
    circs = [C.dd_brickwork(n, depth, np.random.default_rng(C.SEED_BASE + 7000 + i)) for i in range(circuits)]
    dev = []  # per circuit: list of (k, sites, d_sites, d_hi, d_lo)
    for layers in circs:
        steps_c = []
        for layer in layers:
            by_d = {}
            for site, Uh, Ul in layer:
                by_d.setdefault(Uh.shape[0], []).append((site, Uh, Ul))
            for d in sorted(by_d):
                g = by_d[d]
                sites = [s for s, _, _ in g]
                steps_c.append(({2: 1, 4: 2}[d], sites, torch.tensor(sites, dtype=torch.int32, device="cuda"),
                                torch.from_numpy(np.stack([u for _, u, _ in g])).cuda(),
                                torch.from_numpy(np.stack([l for _, _, l in g])).cuda()))
        dev.append(steps_c)
    streams = [torch.cuda.Stream() for _ in range(circuits)]
    hs = [MPSDD(n, chi, cutoff, stream=streams[i]) for i in range(circuits)]

    def one_step():
        for h in hs:
            h.reset()
        for li in range(len(dev[0])):
            for h, steps_c in zip(hs, dev):
                k, sites, d_s, d_hi, d_lo = steps_c[li]
                h.apply_layer_device(sites, d_s, d_hi, k, d_lo)
        for h in hs:
            h.sync()

    one_step()  # warm-up
    ts, flops, upd = [], 0.0, 0
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one_step()
        ts.append(time.perf_counter() - t0)
        for h in hs:
            st = h.stats()
            flops += st["flops"]
            upd += st["updates"]
    t = sum(ts)
    tflops = flops / t / 1e12
    chi_end = hs[0].bond_dims()
    for h in hs:
        h.close()
    # accuracy against the oracle in binary128 (n = 8, depth 8, chi_max = 16)
    nsm = 8
    small = C.dd_brickwork(nsm, 8, np.random.default_rng(C.SEED_BASE + 7999))
    m = MPSDD(nsm, 16, cutoff)
    o = oracle.OracleMPS(nsm, 16, cutoff, oracle.BINARY128)
    for layer in small:
        by_d = {}
        for site, Uh, Ul in layer:
            by_d.setdefault(Uh.shape[0], []).append((site, Uh, Ul))
            o.apply_gate_hl(site, Uh, Ul)
        for d in sorted(by_d):
            g = by_d[d]
            m.apply_layer([s for s, _, _ in g], np.stack([u for _, u, _ in g]), np.stack([l for _, _, l in g]))
    err = 0.0
    for b in range(nsm - 1):
        hi, lo = m.schmidt(b)
        ohi, olo = o.schmidt_hl(b)
        if len(hi) != len(ohi):
            err = float("inf")
            break
        err = max(err, float(np.max(np.abs((hi - ohi) + (lo - olo))) / ohi[0]))
    m.close()
    return {"workload": "%d circuits: n=32, depth-%d Haar U(4) brickwork + RZ, chi_max=32, cutoff 1e-28, "
                        "gates unitary to 1e-32 (hi + lo)" % (circuits, depth),
            "value": upd / t, "unit": "updates/s", "steps": steps, "warmup": 1, "updates_per_step": upd // steps,
            "max_bond": int(chi_end.max()), "timing": "wall clock around the layers of all circuits + sync",
            "executed_binary64_tflops": tflops, "peak_fp64_tflops": fp64_peak_tflops,
            "frac_of_fp64_peak": tflops / fp64_peak_tflops, "peak_source": "derived from unit counts",
            "oracle_binary128_spectrum_err": err,
            "oracle_case": "n=8, depth-8 brickwork + RZ, chi_max=16: max |d lambda| / lambda_0 over all bonds"}


def run_hermitian(fp64_peak_tflops: float, count: int = 4096, spins: int = 5, N: int = 2048):
    """The matrix library's second workload (Sec. 2.1's NMR example, batched):
    `count` strongly coupled `spins`-spin systems (D = 2^spins): thermal state
    (its deviation from I/D) at 300 K, Y_90 pulse on every spin, record of the total X magnetisation
    (N samples, dt = 0.25 ms), zero padding to 2N and |DFT|, every step on the
    GPU; the Jacobi eigensolver's executed flops from its rotation count."""
    import torch
    from oracle import hermitian as O
    from paper_1111_3124_gb300 import circuits as C
    from paper_1111_3124_gb300.mps import dft_abs, fid, heev, hermitian_last_stats, thermal_deviation
    D = 1 << spins
    H = C.spin_hamiltonians(count, spins, np.random.default_rng(C.SEED_BASE + 8000))
    P = C.kron_all(*[C.Y90] * spins)
    Ox = sum(C.kron_all(*[C.X if q == k else C.I2 for q in range(spins)]) for k in range(spins))
    Hd = torch.from_numpy(H).cuda()
    H2 = (2 * np.pi) * Hd
    Pd = torch.from_numpy(np.broadcast_to(P, H.shape).copy()).cuda()
    Od = torch.from_numpy(np.broadcast_to(Ox, H.shape).copy()).cuda()
    beta = C.PLANCK / C.BOLTZMANN / 300.0
    dt = 2.5e-4

    def pipeline():
        # rho - I/D: the record of the traceless X_total depends on it alone,
        # and at 300 K it sits in the 10th digit of rho's entries
        rho = thermal_deviation(Hd, beta)
        s = fid(rho, H2, Od, dt, N, P=Pd)
        return rho, s, dft_abs(s, 2 * N)

    pipeline()  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rho, s, spec = pipeline()
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    heev(Hd)
    torch.cuda.synchronize()
    t_heev = time.perf_counter() - t0
    st = hermitian_last_stats()
    flops = st["rotations"] * (60.0 * D + 25.0)
    # accuracy against the oracle on the first 4 systems
    rho_h, s_h, sp_h = rho[:4].cpu().numpy(), s[:4].cpu().numpy(), spec[:4].cpu().numpy()
    ms = [0, 1, N // 2, N - 1]
    err_rho = err_fid = err_dft = 0.0
    for b in range(4):
        r_ref = O.thermal_deviation(H[b], beta)
        err_rho = max(err_rho, float(np.max(np.abs(rho_h[b] - r_ref)) / np.max(np.abs(r_ref))))
        f_ref = O.fid(r_ref, 2 * np.pi * H[b], Ox, dt, ms, P=P)
        err_fid = max(err_fid, float(np.max(np.abs(s_h[b, ms] - f_ref)) / np.max(np.abs(f_ref))))
        d_ref = O.dft_abs(s_h[b], 2 * N)
        err_dft = max(err_dft, float(np.max(np.abs(sp_h[b] - d_ref)) / np.max(d_ref)))
    return {"workload": "%d strongly coupled %d-spin systems (D=%d), 300 K, Y90 pulses, <X_total> record N=%d, "
                        "zero-padded |DFT| of 2N" % (count, spins, D, N),
            "value": count / t_all, "unit": "systems/s", "seconds_pipeline": t_all, "seconds_heev": t_heev,
            "heev": {"kernel": "k_heev (batched two-sided Jacobi, binary64)", "max_sweeps": st["max_sweeps"],
                     "rotations": st["rotations"], "executed_tflops": flops / t_heev / 1e12,
                     "peak_fp64_tflops": fp64_peak_tflops, "frac": flops / t_heev / 1e12 / fp64_peak_tflops,
                     "peak_source": "derived from unit counts",
                     "flops_per_rotation": "60 D + 25"},
            "oracle_err": {"thermal_deviation_rel": err_rho, "fid_rel": err_fid, "dft_rel": err_dft, "systems": 4},
            "timing": "wall clock around the calls (each synchronises)"}


def run_gpu(a):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1111_3124_gb300 import build as B
    if rank == 0:
        B.build()
    barrier()
    B.build()
    from paper_1111_3124_gb300.mps import MPS, PREC_FP64, PREC_SPLIT, Program

    c, layers, nup = workload()
    glayers = grouped(layers)
    dev_layers = [(k, s, torch.from_numpy(U).to("cuda")) for k, s, U in glayers]
    stream = torch.cuda.Stream()
    prec = PREC_SPLIT if a.prec == "split" else PREC_FP64
    m = MPS(c["n"], c["chi_max"], c["cutoff"], prec)
    m.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step_eager(mm):
        mm.reset()
        for k, s, dU in dev_layers:
            mm.apply_layer_device(s, dU, k)

    # launch shapes of the fp32 sweeps per width: the cached tuner table, else tuned now
    from paper_1111_3124_gb300 import tuner
    tune_table = tuner.load() if not a.retune else None
    tune_source = "cache " + tuner.cache_path()
    if tune_table is None:
        tune_table, _ = tuner.tune()
        tuner.save(tune_table, _)
        tune_source = "tuned in this run (" + tuner.cache_path() + ")"
    m.set_tuning(tune_table)

    with torch.cuda.stream(stream):
        prog = Program([m], program_passes(dev_layers)) if a.path == "program" else None

        def step_device():
            if prog is None:
                step_eager(m)
            else:
                m.reset()
                prog.run()

        for _ in range(a.warmup):
            step_device()
        m.sync()
        try:
            nominal = step_nominal_flops(m, dev_layers, c["n"])
        except Exception:  # a diagnostic only: the bench line does not depend on it
            nominal = None
        chi = m.bond_dims()
        barrier()
        # ---- device-resident timed region
        times = []
        with ClockSampler(local) as clk:
            for _ in range(a.steps):
                flush.fill_(float(len(times)))  # evict L2 between steps
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                step_device()
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
        clocks = clk.summary()
        m.sync()
        # ---- per-kernel-class durations: CUDA events around every launch of
        # one eager step on the same stream (a graph replay cannot be bracketed
        # per kernel); the same kernels at the same sizes as the timed steps
        flush.fill_(0.5)
        m.profile(True)
        t_prof0 = time.perf_counter()
        step_eager(m)
        m.sync()
        t_prof = time.perf_counter() - t_prof0
        prof = {kk: m.profile_read(kk) for kk in range(len(KERNEL_CLASSES))}
        m.profile(False)
        # ---- end to end through the public API with host buffers
        pinned = [(k, s, torch.from_numpy(U).pin_memory().numpy()) for k, s, U in glayers]
        h2d = int(sum(U.nbytes + s.nbytes for _, s, U in pinned))
        mid = c["n"] // 2 - 1
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(a.steps):
            m.reset()
            for k, s, U in pinned:
                m.apply_layer(s, U)
            lam = m.schmidt(mid)
            d2h = lam.nbytes + 4
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0

    # ---- the native binary64 path on the same workload and the split
    # result's deviation from it
    fp64 = None
    if a.prec == "split" and not a.no_fp64_compare:
        with torch.cuda.stream(stream):
            m2 = MPS(c["n"], c["chi_max"], c["cutoff"], PREC_FP64)
            m2.set_stream(stream)
            prog64 = Program([m2], program_passes(dev_layers)) if a.path == "program" else None

            def step64():
                if prog64 is None:
                    step_eager(m2)
                else:
                    m2.reset()
                    prog64.run()

            step64()
            m2.sync()
            t64s = []
            for _ in range(a.fp64_steps):
                flush.fill_(-1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                step64()
                e1.record(stream)
                torch.cuda.synchronize()
                t64s.append(e0.elapsed_time(e1) / 1e3)
            t64 = sum(t64s) / len(t64s)
            bits = np.random.default_rng(11).integers(0, 2, size=(256, c["n"])).astype(np.uint8)
            a_sp, a_64 = m.amplitudes(bits), m2.amplitudes(bits)
            spec = max(float(np.max(np.abs(m.schmidt(b) - m2.schmidt(b)))) / float(np.max(m2.schmidt(b)))
                       if len(m.schmidt(b)) == len(m2.schmidt(b)) else float("inf") for b in range(c["n"] - 1))
            fp64 = {"value": nup / t64, "unit": "updates/s", "ms_per_step": 1e3 * t64, "steps": len(t64s),
                    "warmup": 1, "step_ms": [1e3 * t for t in t64s], "split_speedup": None,
                    "split_vs_fp64": {"max_abs_amp_err": float(np.max(np.abs(a_sp - a_64))),
                                      "max_rel_amp_err": float(np.max(np.abs(a_sp - a_64)) / np.max(np.abs(a_64))),
                                      "max_spectrum_err": spec, "amplitudes_sampled": int(len(bits))}}
            if prog64 is not None:
                prog64.close()
            m2.close()

    t_step = sum(times) / len(times) / 1e3
    t_e2e = e2e_s / a.steps
    t_step, t_e2e = reduce_max([t_step, t_e2e], world)
    value = job_throughput(nup, world, t_step)
    e2e_value = job_throughput(nup, world, t_e2e)

    pk = peaks()
    alu = measure_alu_peaks()
    # ALU-bound kernels are held against the peak derived from the unit counts
    # and the maximum SM clock; the measured library-GEMM throughputs are
    # reported beside them (alu_peaks)
    derived = "derived from unit counts: 152 SMs x %s FMA/clk x 2 flops x %.0f MHz"
    roof_def = {  # class -> (kernel, bound, peak TFLOP/s, peak source)
        0: ("k_jacobi_pair<8,double> (blocked one-sided Jacobi, binary64)", "alu", pk["fp64_tflops"],
            derived % (2, pk["sm_mhz"])),
        1: ("k_contract (theta, binary64)", "alu", pk["fp64_tflops"], derived % (2, pk["sm_mhz"])),
        3: ("k_oz_gemm (split-precision bf16 tcgen05 GEMM)", "tensor", pk["bf16_tflops"], pk["bf16_source"]),
        4: (f32_kernel_name(tune_table, 2 * c["chi_max"]), "alu", pk["fp32_tflops"],
            derived % (128, pk["sm_mhz"])),
    }
    dom = max(roof_def, key=lambda i: prof[i]["ms"])
    d = prof[dom]
    executed = d["flops"] / (d["ms"] / 1e3) / 1e12 if d["ms"] > 0 else None
    name, bound, peak, src = roof_def[dom]
    # algorithmic work: the nominal SVD count of every update of the step
    # charged to the dominant Jacobi kernel's time (its launches carry the
    # SVD); for the tensor-core GEMM its slice products are the algorithm
    if dom in (0, 4) and nominal is not None and d["ms"] > 0:
        achieved = nominal["svd"] / (d["ms"] / 1e3) / 1e12
        algorithmic = ("Golub-Reinsch count 4 (14 M N^2 + 8 N^3) of every update's M x N SVD in one step "
                       "(%.1f GFLOP), over this kernel class's time per step" % (nominal["svd"] / 1e9))
    else:
        achieved = executed
        algorithmic = "tensor-core flops of the slice products"
    # DRAM bytes per launch from one ncu capture of a saturated chi=256 layer
    # (the --profile-layer case), scaled to this run's average launch by
    # duration (the Jacobi kernels are ALU-bound: time tracks work)
    captured = {0: (390.9e6, 2.2237)}
    if f32_mode(tune_table, 2 * c["chi_max"])[1] in F32_CAPTURED:
        captured[4] = F32_CAPTURED[f32_mode(tune_table, 2 * c["chi_max"])[1]]
    ms_launch = d["ms"] / max(d["launches"], 1)
    traffic = captured[dom][0] * ms_launch / captured[dom][1] if dom in captured else None
    roof = {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None, "peak_source": src, "achieved_is": algorithmic,
            "algorithmic_flops_per_launch": achieved * 1e12 * (d["ms"] / 1e3) / max(d["launches"], 1)
            if achieved else None,
            "executed": {"tflops": executed, "frac": executed / peak if executed else None,
                         "flops_per_launch": d["flops"] / max(d["launches"], 1),
                         "counted": "flops executed, counted on the device (Gram, inner rotations, column "
                                    "rotations)" if dom in (0, 4) else "tensor-core flops of the slice products"},
            "ms_per_launch": ms_launch, "traffic": traffic,
            "traffic_source": "ncu dram__bytes_read+write of a saturated launch, scaled by duration"
            if traffic is not None else None,
            "timing": "CUDA events around every launch of one eager step on the handle's stream",
            "share_of_step": d["ms"] / (1e3 * t_prof)}
    kernels = {name: {"ms_per_step": prof[i]["ms"], "launches_per_step": prof[i]["launches"],
                      "tflops": prof[i]["flops"] / (prof[i]["ms"] / 1e3) / 1e12 if prof[i]["ms"] > 0 else None}
               for i, name in enumerate(KERNEL_CLASSES)}
    line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if a.prec == "fp64" else "f64 (bf16 slices + fp32 sweeps)",
            "data": "synthetic (seeded Haar U(4) brickwork + RZ)",
            "config": {"workload": c["name"], "n": c["n"], "depth": c["depth"], "chi_max": c["chi_max"],
                       "cutoff": c["cutoff"], "updates_per_step": nup, "prec": a.prec,
                       "path": "recorded program (one CUDA graph per step)" if a.path == "program"
                       else "eager (host-driven passes)",
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "256 MiB buffer written between timed steps; working set > L2",
                       "tuning": {"table (nw_max, fp32 block, launch mode: 0 per round, 1 tensor-core rotation, "
                                  "2 scheduled, 3 scheduled 384-thread CTAs)": tune_table,
                                  "source": tune_source},
                       "max_bond": int(max(chi)) if len(chi) else 1},
            "roofline": roof, "kernels": kernels, "clocks": clocks,
            "alu_peaks": {"measured": alu, "from_unit_counts": {"fp32_tflops": pk["fp32_tflops"],
                                                                 "fp64_tflops": pk["fp64_tflops"]}},
            "e2e": {"value": e2e_value, "unit": "updates/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "path": "mps_apply_layer with host gates (eager), D2H of the middle bond's Lambda"},
            "gpu_launches": int(prof[0]["launches_all"])}
    if fp64 is not None:
        fp64["split_speedup"] = value / world / fp64["value"]
        line["fp64_path"] = fp64
    if nominal:
        # nominal binary64 work (theta GEMM + Golub-Reinsch SVD count) per second:
        # what a binary64 Golub-Reinsch SVD path would have to sustain to match
        nt = nominal["total"]
        line["nominal_binary64"] = {
            "gflop_per_step": nt / 1e9, "svd_gflop_per_step": nominal["svd"] / 1e9, "tflops": nt / t_step / 1e12,
            "peak_fp64_tflops": alu["fp64_tflops"], "frac_of_fp64_peak": nt / t_step / 1e12 / alu["fp64_tflops"],
            "peak_source": "measured binary64 GEMM throughput",
            "definition": "reference-algorithm-equivalent rate, not executed flops: per update 8*M*N*chi + "
                          "4*(14*M*N^2 + 8*N^3), theta M x N = 2chi_L x 2chi_R"}
        if fp64 is not None:
            fp64["nominal_binary64_tflops"] = nt / (fp64["ms_per_step"] / 1e3) / 1e12
    if rank == 0 and world == 1:
        if not a.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_obj(a.cpu_sample)
            line["oracle_check"] = {"split": oracle_check(PREC_SPLIT, a.cpu_sample),
                                    "fp64": oracle_check(PREC_FP64, a.cpu_sample)}
        if not a.no_extra_configs:
            line["three_site"] = run_three_site(prec, 2, tune_table)
            line["many_circuits"] = run_many_circuits(prec, a.batch_circuits, 1, tune_table)
            line["routing"] = run_routing(prec, tune_table)
            line["double_word"] = run_dd(pk["fp64_tflops"])
            line["hermitian"] = run_hermitian(pk["fp64_tflops"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if prog is not None:
        prog.close()
    m.close()
    if world > 1:
        dist.destroy_process_group()


# fp32 sweeps: DRAM read + write bytes and duration of one captured launch of
# the saturated chi=256 layer (--profile-layer), per launch mode
F32_CAPTURED = {0: (146.0e6, 0.1697), 2: (32.87e9, 47.86)}


def f32_mode(tune_table, nw):
    """(block width, launch mode) the tuning table gives the fp32 sweeps at
    width nw (the library's default without a table: 16, scheduled with
    256-thread CTAs)."""
    bw, mode = 16, 2
    for nw_max, b, md in (tune_table or []):
        bw, mode = b, md
        if nw <= nw_max:
            break
    return bw, mode


def f32_kernel_name(tune_table, nw):
    bw, mode = f32_mode(tune_table, nw)
    if mode in (2, 3):
        return "k_jacobi_f32_sched<%d, %d> (fp32 preconditioning sweeps, one scheduled launch per pass)" % (
            bw, 256 if mode == 2 else 384)
    if mode == 1:
        return "k_jacobi_pair_f32<16> + k_rot_tc (fp32 preconditioning sweeps, tensor-core rotation)"
    return "k_jacobi_pair_f32<%d> (fp32 preconditioning sweeps, one launch per round)" % bw


def run_profile_layer(a):
    """Brickwork layers on a synthetic saturated state (the capture case)."""
    import torch
    from paper_1111_3124_gb300 import build as B
    from paper_1111_3124_gb300 import circuits as C
    torch.cuda.set_device(0)
    B.build()
    from paper_1111_3124_gb300.mps import MPS, PREC_FP64, PREC_SPLIT
    n = a.n or 64
    rng = np.random.default_rng(C.SEED_BASE + 77)
    chi = [1] + [min(a.chi, 2 ** min(b, n - b)) for b in range(1, n)] + [1]
    gammas, lams = C.random_vidal_state(n, chi, rng, decay=2.0)
    m = MPS(n, a.chi, 1e-12, PREC_SPLIT if a.prec == "split" else PREC_FP64)
    m.import_state(gammas, lams)
    nup = 0
    t0 = time.perf_counter()
    for layer in range(a.layers):
        sites = C.brickwork_sites(n, layer)
        Us = np.stack([C.haar_unitary(4, rng) for _ in sites])
        m.apply_layer(sites, Us)
        nup += len(sites)
    m.sync()
    dt = time.perf_counter() - t0
    print("%d updates, %.3f s, max bond %d" % (nup, dt, int(m.bond_dims().max())))
    m.close()


def run_profile_small(a):
    """The capture cases of the double-word path and the Hermitian workload:
    small versions of the `double_word` and `hermitian` lines."""
    import torch
    from paper_1111_3124_gb300 import build as B
    torch.cuda.set_device(0)
    B.build()
    t0 = time.perf_counter()
    if a.profile_dd:
        out = run_dd(1.0, circuits=2, steps=1, depth=8)
    else:
        out = run_hermitian(1.0, count=1024, N=512)
    print("%s: %.3f s, %s %s" % ("double-word" if a.profile_dd else "hermitian", time.perf_counter() - t0,
                                 out["value"], out["unit"]))


def main():
    global ARGS
    a = args_parse()
    ARGS = a
    if a.profile_layer:
        run_profile_layer(a)
        return
    if a.profile_dd or a.profile_hermitian:
        run_profile_small(a)
        return
    if a.impl == "reference":
        import oracle
        oracle.build()
        run_reference(a)
        return
    run_gpu(a)


if __name__ == "__main__":
    main()
