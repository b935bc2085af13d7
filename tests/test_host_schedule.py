"""The block-step schedule's host-side helpers (CPU): next block time and
step levels, compiled from the library's own header with the host compiler.

Every particle keeps a power-of-two step s_i = dt_max 2^-k_i and a time t_i, a
multiple of s_i, with t_i <= t_now < t_i + s_i.  The next block time
min_i (t_i + s_i) is then the next multiple of the smallest occupied step,
which is what block_next_time_q computes from the per-level counts alone.
This checks it against the brute-force minimum over random particle states.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_19294_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r"""
#include "nbody_internal.h"
#include <cstdio>
#include <cstdlib>
// stdin: dt_max dt_min t_now_q n_moved, then 64 level counts; stdout: next time (q)
int main() {
    double dt_max, dt_min;
    long long t_now;
    int moved, lv[64];
    if (scanf("%lf %lf %lld %d", &dt_max, &dt_min, &t_now, &moved) != 4) return 2;
    for (int k = 0; k < 64; ++k)
        if (scanf("%d", &lv[k]) != 1) return 2;
    printf("%lld %d\n", nbody::block_next_time_q(t_now, moved, lv, dt_max, dt_min),
           nbody::block_level(dt_min, dt_max));
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness():
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("no host compiler or CUDA headers")
    d = tempfile.mkdtemp()
    src, exe = os.path.join(d, "h.cpp"), os.path.join(d, "h")
    with open(src, "w") as f:
        f.write(HARNESS)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, "-I", CUDA_INC, src, "-o", exe], check=True)
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def run(exe, dt_max, dt_min, t_now, moved, counts):
    inp = f"{dt_max!r} {dt_min!r} {t_now} {moved} " + " ".join(str(int(c)) for c in counts)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
    return int(out[0]), int(out[1])


def test_next_block_time_is_the_brute_force_minimum(harness):
    rng = np.random.default_rng(11)
    for _ in range(200):
        kmax = int(rng.integers(0, 41))        # dt_max / dt_min up to 2^40
        dt_max = 2.0 ** int(rng.integers(-12, 3))
        dt_min = dt_max * 2.0 ** -kmax
        t_now = int(rng.integers(0, 2 ** 50))  # current block time in units of dt_min
        n = int(rng.integers(1, 40))
        levels = rng.integers(0, kmax + 1, n)
        steps = [1 << (kmax - int(k)) for k in levels]  # in units of dt_min
        nxt = min((t_now // s) * s + s for s in steps)
        counts = np.bincount(levels, minlength=64)
        got, lev = run(harness, dt_max, dt_min, t_now, 1, counts)
        assert lev == kmax
        assert got == nxt, (kmax, t_now, sorted(set(steps)), got, nxt)


def test_a_step_that_moved_nobody_keeps_the_time(harness):
    counts = np.zeros(64, dtype=int)
    counts[3] = 5
    assert run(harness, 2.0 ** -7, 2.0 ** -22, 12345, 0, counts)[0] == 12345


def test_levels_of_power_of_two_steps(harness):
    for kmax in (0, 1, 15, 40):
        got = run(harness, 1.0, 2.0 ** -kmax, 0, 0, np.zeros(64, dtype=int))[1]
        assert got == kmax
