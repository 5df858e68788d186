"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_l2(got, ref):
    """Relative L2 error per estimate vector (last axis)."""
    num = np.linalg.norm(np.asarray(got) - np.asarray(ref), axis=-1)
    den = np.maximum(np.linalg.norm(np.asarray(ref), axis=-1), 1e-30)
    return num / den


def assert_vectors_close(got, ref, tol=1e-4, what=""):
    e = rel_l2(got, ref)
    bad = np.argwhere(e > tol)
    assert bad.size == 0, f"{what}: {bad.shape[0]} vectors above rel L2 {tol:g}; max {e.max():.3e} at {bad[0]}"
    return float(e.max()) if e.size else 0.0


def assert_decisions_match(got, ref, M, margin=1e-3):
    """Hard decisions agree except where the oracle lies within `margin` of a decision threshold."""
    from paper_1902_08653_gb300 import workload as wl

    lg, _ = wl.hard_decision(got, M)
    lr, mr = wl.hard_decision(ref, M)
    keep = mr >= margin
    assert np.array_equal(lg[keep], lr[keep]), f"{int(np.sum(lg[keep] != lr[keep]))} decisions differ"
    return int(np.sum(~keep))


def offsets(cs):
    return np.concatenate([[0], np.cumsum(cs)]).astype(int)
