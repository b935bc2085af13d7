"""Host-side fault injection: a context's allocation cap (GPU).

nbody_config.max_device_bytes caps the device memory a context may hold; an
allocation that would pass it is refused before cudaMalloc is called and fails
the call with NBODY_ENOMEM, the same status a failed cudaMalloc gives.  No
kernel is made to fail: the refusal happens on the host, so the GPU and other
contexts stay usable, which the tests check.
"""
import numpy as np
import pytest
import torch

import paper_2509_19294_gb300 as nb
from paper_2509_19294_gb300 import ic
from tests.gpu_util import dev, forces, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_19294_gb300 import build
    build.build()
    nb.load()
    torch.cuda.init()


def _init_ok(n, cap):
    try:
        nb.nbody_destroy(nb.nbody_init(n, 0.01, max_device_bytes=cap))
        return True
    except nb.NBodyError as e:
        assert e.code == nb.NBODY_ENOMEM, e      # no context is left to carry a message
        return False


def test_cap_refuses_init_and_lazy_state_with_enomem():
    n = 4096
    pos, vel, mass = ic.plummer(n, seed=31)
    ref_a, ref_p = forces(pos, mass, 0.01)
    with pytest.raises(nb.NBodyError) as e:
        nb.nbody_init(n, 0.01, max_device_bytes=1)
    assert e.value.code == nb.NBODY_ENOMEM
    with pytest.raises(nb.NBodyError) as e:
        nb.nbody_init(n, 0.01, max_device_bytes=-1)
    assert e.value.code == nb.NBODY_EINVAL
    # the smallest cap nbody_init accepts (bisection over the cap)
    lo, hi = 1, 1 << 33
    assert _init_ok(n, hi)
    while lo < hi:
        mid = (lo + hi) // 2
        if _init_ok(n, mid):
            hi = mid
        else:
            lo = mid + 1
    cap = lo
    with nb.nbody_init(n, 0.01, max_device_bytes=cap) as ctx:
        p, v, m = dev(pos), dev(vel), dev(mass)
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_forces(ctx, p, m, acc, pot)             # allocates nothing more
        assert np.array_equal(host(acc), ref_a) and np.array_equal(host(pot), ref_p)
        jerk = torch.empty((3, n), dtype=torch.float64, device="cuda")
        with pytest.raises(nb.NBodyError) as e:          # the jerk path is built on first use
            nb.nbody_forces_jerk(ctx, p, v, m, acc, jerk, pot)
        assert e.value.code == nb.NBODY_ENOMEM and "allocation cap" in str(e.value)
        with pytest.raises(nb.NBodyError) as e:          # the error is sticky
            nb.nbody_forces(ctx, p, m, acc, pot)
        assert e.value.code == nb.NBODY_ESTATE
    # host arrays need staging buffers: refused under the same cap
    with nb.nbody_init(n, 0.01, max_device_bytes=cap) as ctx:
        with pytest.raises(nb.NBodyError) as e:
            nb.nbody_forces(ctx, pos, mass, np.empty((3, n)), np.empty(n))
        assert e.value.code == nb.NBODY_ENOMEM
    # the device is unaffected: a context without a cap gives the same result
    a, p_ = forces(pos, mass, 0.01)
    assert np.array_equal(a, ref_a) and np.array_equal(p_, ref_p)
