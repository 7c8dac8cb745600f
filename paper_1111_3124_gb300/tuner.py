"""Per-width tuner of the split mode's fp32 sweeps.

For each bucket of working-matrix widths Nw (the smaller dimension of theta,
2 chi at saturation), times one brickwork layer of Haar U(4) updates on a
synthetic state of 64 sites whose bonds sit at chi = Nw / 2 (where the
chain's ends allow), once per candidate launch
shape (fp32 block width 8 or 16; one launch per round with the block
rotations in the pair kernel or on the tensor cores, or every sweep in one
scheduled launch of 256- or 384-thread CTAs), and keeps the fastest. The table is cached as JSON and applied
to handles with MPS.set_tuning; nothing here computes any part of the update.

  python -m paper_1111_3124_gb300.tuner [--out PATH] [--chis 32 64 128 256]
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

# (fp32 block width, launch mode): 0 one launch per round, rotation in the
# pair kernel; 1 the same with the rotation on the tensor cores; 2 every sweep
# in one scheduled launch of 256-thread CTAs; 3 the same with 384-thread CTAs
CANDIDATES = [(16, 3), (8, 3), (16, 2), (8, 2), (16, 0), (8, 0), (16, 1)]
MODE_NAMES = {0: "round", 1: "tc", 2: "sched", 3: "sched384"}
DEFAULT_CHIS = (32, 64, 128, 256)


def cache_path() -> str:
    return os.environ.get("MPS_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_1111_3124_gb300", "tune.json"))


def _layer_time(chi: int, cand, n: int, reps: int) -> float:
    from . import circuits as C
    from .mps import MPS, PREC_SPLIT
    rng = np.random.default_rng(C.SEED_BASE + 99)
    chis = [1] + [min(chi, 2 ** min(b, n - b)) for b in range(1, n)] + [1]
    gammas, lams = C.random_vidal_state(n, chis, rng, decay=2.0)
    sites = C.brickwork_sites(n, 0)
    Us = np.stack([C.haar_unitary(4, rng) for _ in sites])
    m = MPS(n, chi, 1e-12, PREC_SPLIT)
    m.set_tuning([(4096, cand[0], cand[1])])
    best = float("inf")
    for r in range(reps + 1):
        m.import_state(gammas, lams)
        m.sync()
        t0 = time.perf_counter()
        m.apply_layer(sites, Us)
        m.sync()
        if r:
            best = min(best, time.perf_counter() - t0)
    m.close()
    return best


def tune(chis=DEFAULT_CHIS, reps: int = 3, n: int = 64):
    """Returns (table, measurements): table rows (nw_max, f32_block, mode).
    n = 64 sites give a layer of about 30 concurrent updates, most of them
    saturated, as in the circuits the table serves."""
    table, meas = [], {}
    for chi in chis:
        times = {cand: _layer_time(chi, cand, n, reps) for cand in CANDIDATES}
        best = min(times, key=times.get)
        table.append((2 * chi, best[0], best[1]))
        meas[str(2 * chi)] = {"%d/%s" % (c[0], MODE_NAMES[c[1]]): t for c, t in times.items()}
    return table, meas


def save(table, meas, path: str | None = None) -> str:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump({"table": table, "seconds_per_layer": meas}, f, indent=1)
    return path


def load(path: str | None = None):
    path = path or cache_path()
    try:
        with open(path) as f:
            return [tuple(r) for r in json.load(f)["table"]]
    except (OSError, ValueError, KeyError):
        return None


def main() -> None:
    import argparse
    p = argparse.ArgumentParser()
    p.add_argument("--out", default=None)
    p.add_argument("--chis", type=int, nargs="*", default=list(DEFAULT_CHIS))
    a = p.parse_args()
    from . import build as B
    B.build()
    table, meas = tune(a.chis)
    print(json.dumps({"table": table, "seconds_per_layer": meas, "path": save(table, meas, a.out)}))


if __name__ == "__main__":
    main()
