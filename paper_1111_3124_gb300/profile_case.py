"""One layer of two-site updates on a synthetic saturated state: the case that
hardware-counter captures of the update kernels run on.

A Vidal-form state with every bond at chi (Gamma complex Gaussian, Lambda
descending) gets one brickwork layer of Haar-random U(4) gates, so every
update works on a full 2chi x 2chi theta, as in the steady state of a
saturated simulation, after only a few setup launches.

  python -m paper_1111_3124_gb300.profile_case [--n 64] [--chi 256]
         [--prec split|fp64] [--layers 1]
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import circuits as C


def main() -> None:
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=64)
    p.add_argument("--chi", type=int, default=256)
    p.add_argument("--prec", default="split", choices=["split", "fp64"])
    p.add_argument("--layers", type=int, default=1)
    a = p.parse_args()

    from . import build as B
    B.build()
    from .mps import MPS, PREC_FP64, PREC_SPLIT

    rng = np.random.default_rng(C.SEED_BASE + 77)
    chi = [1] + [min(a.chi, 2 ** min(b, a.n - b)) for b in range(1, a.n)] + [1]
    gammas, lams = C.random_vidal_state(a.n, chi, rng, decay=2.0)
    m = MPS(a.n, a.chi, 1e-12, PREC_SPLIT if a.prec == "split" else PREC_FP64)
    m.import_state(gammas, lams)
    nup = 0
    t0 = time.perf_counter()
    for layer in range(a.layers):
        sites = C.brickwork_sites(a.n, layer)
        Us = np.stack([C.haar_unitary(4, rng) for _ in sites])
        m.apply_layer(sites, Us)
        nup += len(sites)
    m.sync()
    dt = time.perf_counter() - t0
    print(f"{nup} updates, {dt:.3f} s, max bond {int(m.bond_dims().max())}")
    m.close()


if __name__ == "__main__":
    main()
