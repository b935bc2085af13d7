"""Error statistics used by the parity tests (comparison only, no method arithmetic)."""
import numpy as np


def rel_acc_errors(a, ref):
    """Per-particle |a - ref| / |ref| (Euclidean norms over the 3 components)."""
    num = np.linalg.norm(np.asarray(a) - np.asarray(ref), axis=0)
    den = np.linalg.norm(np.asarray(ref), axis=0)
    return num / np.where(den > 0, den, 1.0)


def paper_metric(a, ref):
    """The paper's validation bound (Sec. 3): each acceleration component
    within 0.05 % of a force magnitude it calls typical without defining it.
    Per-particle reading, against the particle's own magnitude:
    max_i,k |a_ik - ref_ik| / |ref_i|."""
    a, ref = np.asarray(a), np.asarray(ref)
    den = np.linalg.norm(ref, axis=0)
    return float((np.abs(a - ref).max(axis=0) / np.where(den > 0, den, 1.0)).max())


def paper_metric_rms(a, ref):
    """The same bound with one global scale, the RMS magnitude as the typical
    one: max_i,k |a_ik - ref_ik| / RMS_i |ref_i|.  Independent of the
    per-particle relative-error gates; a particle in a close encounter
    (|a_i| >> RMS) then needs a relative error below 5e-4 * RMS / |a_i|."""
    typical = np.sqrt(np.mean(np.sum(np.asarray(ref) ** 2, axis=0)))
    return float(np.abs(np.asarray(a) - np.asarray(ref)).max() / typical)


def rel_pot_errors(p, ref):
    return np.abs(np.asarray(p) - np.asarray(ref)) / np.abs(np.asarray(ref))


def summary(a, ref, p=None, pref=None):
    e = rel_acc_errors(a, ref)
    out = {"median": float(np.median(e)), "max": float(e.max()), "paper": paper_metric(a, ref),
           "paper_rms": paper_metric_rms(a, ref)}
    if p is not None:
        ep = rel_pot_errors(p, pref)
        out["pot_median"] = float(np.median(ep))
        out["pot_max"] = float(ep.max())
    return out
