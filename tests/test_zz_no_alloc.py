"""nbody_forces_noalloc, the allocation-free force entry point (GPU).

Some callers cannot allocate device memory when they need forces -- code that
runs inside a memory pool it does not own, loops that must not pay allocation
latency, plug-ins in a process that has reserved the GPU's memory.  For them the
library offers nbody_forces_noalloc, which keeps its scratch in a fixed array
compiled into libnbody.so instead of a context allocated by nbody_init.

These tests call it through the C ABI and check every output element against
the FP64 oracle with the FP32C tolerance of the parity tests (per-particle
relative acceleration error: median <= 1e-6, max <= 1e-4; potential likewise):
two calls in a row with different inputs (the second proves that the shared
scratch is re-initialised), eps = 0 with coincident particles, a size whose
split count is 2, and the largest size the scratch holds (split 1, every tile
of the array in use; sampled rows).  The file is named so that pytest collects
it last; it passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest
import torch

import paper_2509_19294_gb300 as nb
from paper_2509_19294_gb300 import ic
from tests import metrics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_19294_gb300 import build
    build.build()
    nb.load()
    torch.cuda.init()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _assert_close(a, p, ra, rp):
    s = metrics.summary(a, ra, p, rp)
    assert s["median"] <= 1e-6 and s["max"] <= 1e-4, s
    assert s["pot_median"] <= 1e-6 and s["pot_max"] <= 1e-4, s
    return s


def _call(lib, pos, mass, eps, G, stream):
    n = mass.shape[0]
    p, m = _dev(pos), _dev(mass)
    acc = torch.full((3, n), float("nan"), dtype=torch.float64, device="cuda")
    pot = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.nbody_forces_noalloc(n, p.data_ptr(), m.data_ptr(), eps, G, acc.data_ptr(),
                                  pot.data_ptr(), stream)
    assert rc == nb.NBODY_OK, nb.nbody_strerror(rc)
    return p, m, acc, pot                  # the inputs stay alive until the sync


def test_two_calls_in_a_row_match_the_oracle(oracle):
    lib = nb.load()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [
        (ic.plummer(30001, seed=21)[::2], 0.002, 1.0),
        (ic.uniform_sphere(20000, seed=22, masses=ic.log_uniform_masses(20000, 23))[::2], 0.0, 0.7),
    ]
    outs = [_call(lib, pos, mass, eps, G, stream) for (pos, mass), eps, G in cases]
    torch.cuda.synchronize()
    for ((pos, mass), eps, G), (_, _, acc, pot) in zip(cases, outs):
        ra, rp = oracle.forces(pos, mass, eps, G)
        _assert_close(acc.cpu().numpy(), pot.cpu().numpy(), ra, rp)


def test_eps_zero_coincident_particles_match_the_oracle(oracle):
    # with eps = 0 a coincident distinct pair contributes nothing (the oracle
    # skips r = 0 too); every 97th particle is duplicated onto its neighbour
    lib = nb.load()
    stream = torch.cuda.current_stream().cuda_stream
    pos, _, mass = ic.plummer(5000, seed=25)
    pos = pos.copy()
    pos[:, 1::97] = pos[:, 0:-1:97][:, :pos[:, 1::97].shape[1]]
    _, _, acc, pot = _call(lib, pos, mass, 0.0, 1.0, stream)
    torch.cuda.synchronize()
    a, p = acc.cpu().numpy(), pot.cpu().numpy()
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(p))
    ra, rp = oracle.forces(pos, mass, 0.0)
    _assert_close(a, p, ra, rp)


@pytest.mark.parametrize("n", [60000, nb.NBODY_NOALLOC_MAX_N])
def test_split_two_and_full_scratch_sampled_rows(oracle, n):
    # n = 60000: 235 tiles of 256, split 2; n = NBODY_NOALLOC_MAX_N: 1024 tiles,
    # split 1, the queue, counters and packed arrays fill the fixed scratch
    lib = nb.load()
    stream = torch.cuda.current_stream().cuda_stream
    pos, _, mass = ic.plummer(n, seed=26)
    _, _, acc, pot = _call(lib, pos, mass, 1e-3, 1.0, stream)
    torch.cuda.synchronize()
    a, p = acc.cpu().numpy(), pot.cpu().numpy()
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(p))
    rows = np.unique(np.concatenate([ic.sample_rows(n, 1024, 27), [0, n - 1]]))
    ra, rp = oracle.forces_rows(pos, mass, 1e-3, rows)
    _assert_close(a[:, rows], p[rows], ra, rp)


def test_rejects_oversize_and_host_arrays():
    lib = nb.load()
    n = nb.NBODY_NOALLOC_MAX_N + 1
    rc = lib.nbody_forces_noalloc(n, 8, 8, 0.01, 1.0, 8, None, None)
    assert rc == nb.NBODY_ETOOBIG
    assert "NBODY_NOALLOC_MAX_N" in nb.nbody_strerror(rc)
    pos, _, mass = ic.plummer(100, seed=24)
    acc = np.empty((3, 100))
    with pytest.raises(nb.NBodyError) as e:
        nb.nbody_forces_noalloc(pos, mass, 0.01, acc)
    assert e.value.code == nb.NBODY_EINVAL
    assert lib.nbody_forces_noalloc(0, None, None, 0.01, 1.0, None, None, None) == nb.NBODY_OK
