"""Helpers for the GPU tests: torch device arrays and one call to the library."""
import numpy as np
import torch

import paper_2509_19294_gb300 as nb


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def forces(pos, mass, eps, mode=nb.NBODY_F32C, G=1.0, offsets=None, **kw):
    """One nbody_forces call on device arrays; returns (acc, pot) as numpy."""
    n = mass.shape[0]
    with nb.nbody_init(n, eps, mode=mode, G=G, cluster_offsets=offsets, **kw) as ctx:
        p, m = dev(pos), dev(mass)
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_forces(ctx, p, m, acc, pot)
        return host(acc), host(pot)
