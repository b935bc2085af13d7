"""Error statistics used by the parity tests (comparison only, no method arithmetic)."""
import numpy as np


def rel_acc_errors(a, ref):
    """Per-particle |a - ref| / |ref| (Euclidean norms over the 3 components)."""
    num = np.linalg.norm(np.asarray(a) - np.asarray(ref), axis=0)
    den = np.linalg.norm(np.asarray(ref), axis=0)
    return num / np.where(den > 0, den, 1.0)


def paper_metric(a, ref):
    """max_i,k |a_ik - ref_ik| / RMS_i |ref_i|: the paper's "fraction of a typical
    force magnitude" (Sec. 3 validation paragraph), typical read as the RMS."""
    typical = np.sqrt(np.mean(np.sum(np.asarray(ref) ** 2, axis=0)))
    return np.abs(np.asarray(a) - np.asarray(ref)).max() / typical


def rel_pot_errors(p, ref):
    return np.abs(np.asarray(p) - np.asarray(ref)) / np.abs(np.asarray(ref))


def summary(a, ref, p=None, pref=None):
    e = rel_acc_errors(a, ref)
    out = {"median": float(np.median(e)), "max": float(e.max()), "paper": float(paper_metric(a, ref))}
    if p is not None:
        ep = rel_pot_errors(p, pref)
        out["pot_median"] = float(np.median(ep))
        out["pot_max"] = float(ep.max())
    return out
