"""The block-step force pass's even split of its work (CPU), compiled from the
library's own header with the host compiler.

The F32C subset kernels take the step's (i-chunk, j-tile) units in unit order
(clusters, their i-chunks, the j-tiles), cut into one contiguous range per
CTA.  A CTA finalises the i-chunks its range covers whole and writes a partial
for each one it shares, to a slot it derives from its own range; the tail
kernel finds the ranges that share a chunk, and their slots, from the chunk's
first unit alone.  The two sides use the header's even_range_begin,
even_range_of and even_range_slot.  This checks, over random layouts and range
counts, that the ranges partition the units, that every shared chunk's writers
are exactly the ranges and slots its reader sums, in range order, and that no
slot is written twice.
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

# stdin: n_ranges n_chunks, then each chunk's j-tile count.  stdout: one line
# per range (its first and end unit), then per chunk the writers as the CTAs
# see them ("W chunk range slot", in range order; "F chunk range" for a chunk a
# range covers whole) and the readers as the tail sees them ("R chunk range
# slot" for a shared chunk).
HARNESS = r"""
#include "nbody_internal.h"
#include <cstdio>
#include <vector>
using namespace nbody;
int main() {
    long long nr, nc;
    if (scanf("%lld %lld", &nr, &nc) != 2) return 2;
    std::vector<long long> njt(nc), first(nc + 1, 0);
    for (long long c = 0; c < nc; ++c) {
        if (scanf("%lld", &njt[c]) != 1) return 2;
        first[c + 1] = first[c] + njt[c];
    }
    const long long W = first[nc];
    for (long long r = 0; r < nr; ++r)
        printf("B %lld %lld %lld\n", r, even_range_begin(r, W, nr), even_range_begin(r + 1, W, nr));
    // the CTAs: each walks its range chunk by chunk, as the subset kernel does
    for (long long r = 0; r < nr; ++r) {
        const long long u0 = even_range_begin(r, W, nr), u1 = even_range_begin(r + 1, W, nr);
        long long c = 0;
        for (long long u = u0; u < u1;) {
            while (first[c + 1] <= u) ++c;
            const long long t = u - first[c];
            const long long t1 = njt[c] < t + (u1 - u) ? njt[c] : t + (u1 - u);
            if (t == 0 && t1 == njt[c]) printf("F %lld %lld\n", c, r);
            else printf("W %lld %lld %lld\n", c, r, even_range_slot(r, u - t, W, nr));
            u += t1 - t;
        }
    }
    // the tail: per chunk, the ranges from its first unit
    for (long long c = 0; c < nc; ++c) {
        const long long uc = first[c];
        const long long wa = even_range_of(uc, W, nr), wb = even_range_of(uc + njt[c] - 1, W, nr);
        if (wa == wb) continue;
        for (long long r = wa; r <= wb; ++r) printf("R %lld %lld %lld\n", c, r, even_range_slot(r, uc, W, nr));
    }
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


def run(exe, n_ranges, njt):
    inp = f"{n_ranges} {len(njt)} " + " ".join(str(int(x)) for x in njt)
    lines = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    rec = {"B": [], "F": [], "W": [], "R": []}
    for ln in lines:
        if ln:
            k, *v = ln.split()
            rec[k].append(tuple(int(x) for x in v))
    return rec


def check(rec, n_ranges, njt):
    W = int(np.sum(njt))
    # the ranges partition the units, each at least one unit when W >= n_ranges
    ends = [b for b in rec["B"]]
    assert ends[0][1] == 0 and ends[-1][2] == W
    for (r, b, e), (_, b2, _) in zip(ends, ends[1:]):
        assert e == b2
    assert all(e > b for _, b, e in ends) or W < n_ranges
    # a chunk is either covered whole by one range or shared; the writers of a
    # shared chunk are exactly its readers, in range order, with the same slots
    full = {c for c, _ in rec["F"]}
    writers, readers = {}, {}
    for c, r, slot in rec["W"]:
        writers.setdefault(c, []).append((r, slot))
    for c, r, slot in rec["R"]:
        readers.setdefault(c, []).append((r, slot))
    assert not (full & set(writers)), "a chunk both finalised whole and shared"
    assert set(full) | set(writers) == set(range(len(njt)))
    assert writers == readers
    # the tail takes every range after a shared chunk's first one to start
    # inside the chunk and adds its slot 2r without asking the header again
    for c, rs in readers.items():
        assert all(slot == 2 * r for r, slot in rs[1:]), (c, rs)
    slots = [s for _, _, s in rec["W"]]
    assert len(slots) == len(set(slots)), "a partial slot written twice"
    assert all(0 <= s < 2 * n_ranges for s in slots)


def test_even_split_writers_and_readers_agree(harness):
    rng = np.random.default_rng(17)
    for _ in range(300):
        n_chunks = int(rng.integers(1, 60))
        njt = rng.integers(1, 50, n_chunks)
        W = int(njt.sum())
        n_ranges = int(rng.integers(1, max(2, W // 2) + 1))  # at least two units a range, as planned
        check(run(harness, n_ranges, njt), n_ranges, njt)


def test_even_split_at_the_bench_shapes(harness):
    # the N = 102 400 block-step regimes: 400 j-tiles a chunk, 304 or 608 ranges
    for n_chunks, n_ranges in ((1, 152), (2, 304), (8, 304), (14, 608), (41, 608), (800, 608)):
        njt = np.full(n_chunks, 400)
        check(run(harness, n_ranges, njt), n_ranges, njt)
