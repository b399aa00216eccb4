"""Shared helpers of the test suite: turning a seeded workload into the inputs
of each side.  Each side converts Kipping's (q1, q2) with its own code: the
product through gl_q_to_u, the oracle through oracle.q_to_u."""
import numpy as np

from paper_2410_05408_b300 import inputs

PARAM_NAMES = inputs.PARAM_NAMES


def product_params(wl):
    """float64 parameter arrays for the library (u from gl_q_to_u)."""
    from paper_2410_05408_b300 import binding
    p = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in wl["params"].items()}
    if "u1" not in p:
        p["u1"], p["u2"] = binding.gl_q_to_u(p.pop("q1"), p.pop("q2"))
    return {k: p[k] for k in PARAM_NAMES}


def oracle_params(wl, idx=None):
    """float64 parameter arrays for the oracle (u from oracle.q_to_u)."""
    import oracle
    p = {k: np.asarray(v, dtype=np.float64) for k, v in wl["params"].items()}
    if "u1" not in p:
        u = np.array([oracle.q_to_u(a, b) for a, b in zip(p.pop("q1"), p.pop("q2"))])
        p["u1"], p["u2"] = u[:, 0].copy(), u[:, 1].copy()
    if idx is not None:
        p = {k: v[idx] for k, v in p.items()}
    return {k: p[k] for k in PARAM_NAMES}


def nsuper_array(wl, n_sets):
    ns = wl["nsuper"]
    if np.ndim(ns) == 0:
        return np.full(n_sets, int(ns), dtype=np.int32)
    return np.ascontiguousarray(ns, dtype=np.int32)
