"""Shared test helpers (numpy only; no method arithmetic beyond re-contracting
exported tensors for gauge-invariant comparisons)."""
import numpy as np

import oracle
from paper_1111_3124_gb300 import circuits as C


def all_bits(n):
    return np.array([[(x >> (n - 1 - q)) & 1 for q in range(n)] for x in range(1 << n)], dtype=np.uint8)


def oracle_run(n, layers, chi_max, cutoff, prec=oracle.FP64, state=None):
    m = oracle.OracleMPS(n, chi_max, cutoff, prec)
    if state is not None:
        m.set_state(*state)
    for layer in layers:
        for site, U in layer:
            m.apply_gate(site, U)
    return m


def two_site_tensor(gammas, lams, s):
    """theta~[(i,a),(j,b)] = L_{s-1}[a] G_s[i,a,c] L_s[c] G_{s+1}[j,c,b] L_{s+1}[b]:
    gauge invariant when the spectrum has a gap at the cut."""
    n = len(gammas)
    lam = lambda b: np.ones(1) if b < 0 or b >= n - 1 else lams[b]
    G0, G1 = gammas[s], gammas[s + 1]
    t = np.einsum("a,iac,c,jcb,b->iajb", lam(s - 1), G0, lam(s), G1, lam(s + 1))
    return t.reshape(2 * G0.shape[1], 2 * G1.shape[2])


def three_site_tensor(gammas, lams, s):
    n = len(gammas)
    lam = lambda b: np.ones(1) if b < 0 or b >= n - 1 else lams[b]
    G0, G1, G2 = gammas[s], gammas[s + 1], gammas[s + 2]
    t = np.einsum("a,iac,c,jcd,d,ldb,b->iajlb", lam(s - 1), G0, lam(s), G1, lam(s + 1), G2, lam(s + 2))
    return t.reshape(2 * G0.shape[1], 4 * G2.shape[2])


def spectrum_err(a, b):
    """max |d lambda| / lambda_0 over the common length; lengths must agree."""
    assert len(a) == len(b), (len(a), len(b))
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def random_state(n, chi, seed):
    return C.random_vidal_state(n, chi, np.random.default_rng(seed))
