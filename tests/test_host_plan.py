"""The block-step planner (CPU), compiled from the library's own header with
the host compiler.

plan_step runs in one thread after the scan of the per-unit active counts
(F32C: centre tiles; FP64: row chunks) and decides the step: each cluster's
active range and i-chunk count, the regime (few-particle pass, small-set or
large-set subset kernel) and the force pass's work -- for F32C the
(i-chunk, j-tile) units cut into even ranges, one per CTA; for the FP64 path
queue items of (i-chunk, j-range).  This checks its outputs against their
definitions over random layouts: the active ranges are the scan's, the chunk
counts the ceilings, the regime the thresholds, the F32C range count at most
the CTA count, a multiple of the SM count once above it, with at least two
units a range, and the few-particle lists the active clusters in order.
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

# stdin: f32c ncl n_units; per cluster n n_jt unit_first; unit_first[ncl];
# per unit its active count; then cs_small workers_small max_split few_max
# cs_large workers_large large_min sms.  stdout: the plan.
HARNESS = r"""
#include "nbody_internal.h"
#include <cstdio>
#include <cstring>
#include <vector>
using namespace nbody;
int main() {
    int f32c, ncl, nu;
    if (scanf("%d %d %d", &f32c, &ncl, &nu) != 3) return 2;
    std::vector<ClusterDev> cl(ncl);
    std::vector<int32_t> first(ncl + 1);
    for (int c = 0; c < ncl; ++c) {
        memset(&cl[c], 0, sizeof(ClusterDev));
        int n, njt;
        if (scanf("%d %d %d", &n, &njt, &first[c]) != 3) return 2;
        cl[c].n = n;
        cl[c].n_jt = njt;
    }
    if (scanf("%d", &first[ncl]) != 1) return 2;
    std::vector<int> cnt(nu), off(nu);
    int total = 0;
    for (int u = 0; u < nu; ++u) {
        if (scanf("%d", &cnt[u]) != 1) return 2;
        off[u] = total;
        total += cnt[u];
    }
    int cs_small, workers_small, max_split, few_max, cs_large, workers_large, large_min, sms;
    if (scanf("%d %d %d %d %d %d %d %d", &cs_small, &workers_small, &max_split, &few_max, &cs_large,
              &workers_large, &large_min, &sms) != 8) return 2;
    std::vector<int> act_begin(ncl + 1), act_n(ncl + 1), ich_off(ncl + 1), item_off(ncl + 1);
    std::vector<long long> work_off(ncl + 1);
    BlockScalars sc;
    memset(&sc, 0, sizeof sc);
    plan_step(off.data(), total, nu, first.data(), ncl, cl.data(), cs_small, workers_small, max_split,
              act_begin.data(), act_n.data(), ich_off.data(), item_off.data(), &sc, few_max, cs_large,
              workers_large, large_min, 1LL << 40, f32c ? work_off.data() : nullptr, sms);
    printf("S %d %d %d %d %d %d %d %d %lld %d %lld %lld\n", sc.n_active, sc.few, sc.few_ncl, sc.n_chunks,
           sc.split, sc.n_items, sc.cs, sc.n_items_small, (long long)sc.n_items_large, sc.n_workers,
           sc.n_units, sc.blocks);
    for (int c = 0; c < ncl; ++c)
        printf("C %d %d %d %d %lld\n", act_begin[c], act_n[c], ich_off[c], item_off[c], work_off[c]);
    printf("E %d %d %lld\n", ich_off[ncl], item_off[ncl], work_off[ncl]);
    for (int k = 0; k < sc.few_ncl; ++k) printf("F %d %d %d\n", sc.few_cl[k], sc.few_abeg[k], sc.few_jbase[k]);
    printf("J %d\n", sc.few_jbase[sc.few_ncl]);
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


P = dict(cs_small=64, workers_small=304, max_split=128, few_max=32, cs_large=128, workers_large=608,
         large_min=512, sms=152)


def plan(exe, f32c, ns, njt, first, counts, p=P):
    inp = [f"{int(f32c)} {len(ns)} {len(counts)}"]
    inp += [f"{n} {j} {f}" for n, j, f in zip(ns, njt, first[:-1])]
    inp += [str(first[-1]), " ".join(str(int(c)) for c in counts)]
    inp += [" ".join(str(p[k]) for k in ("cs_small", "workers_small", "max_split", "few_max", "cs_large",
                                         "workers_large", "large_min", "sms"))]
    out = subprocess.run([exe], input="\n".join(inp), capture_output=True, text=True, check=True).stdout
    rec = {"S": None, "C": [], "E": None, "F": [], "J": None}
    for ln in out.splitlines():
        k, *v = ln.split()
        v = [int(x) for x in v]
        if k in ("C", "F"):
            rec[k].append(v)
        else:
            rec[k] = v
    return rec


def layout(rng, ncl, tile, tj, nmax):
    ns = rng.integers(1, nmax, ncl)
    tiles = (ns + tile - 1) // tile
    first = np.concatenate([[0], np.cumsum(tiles)])
    njt = (ns + tj - 1) // tj
    return ns, njt, first


def check(rec, f32c, ns, njt, first, counts, p=P):
    (n_active, few, few_ncl, n_chunks, split, n_items, cs, small, large_items, n_workers, n_units,
     blocks) = rec["S"]
    total = int(np.sum(counts))
    assert n_active == total and blocks == (1 if total > 0 else 0)
    want_few = 0 < total <= p["few_max"]
    want_large = not want_few and total >= p["large_min"]
    assert few == int(want_few)
    assert cs == (p["cs_large"] if want_large else p["cs_small"])
    ncl = len(ns)
    chunks = 0
    for c in range(ncl):
        a0, an, ich, _, _ = rec["C"][c]
        assert a0 == int(np.sum(counts[:first[c]])) and an == int(np.sum(counts[first[c]:first[c + 1]]))
        assert ich == chunks
        if not want_few:
            chunks += -(-an // cs)
    assert rec["E"][0] == chunks == n_chunks
    # the few-particle lists: the clusters holding active particles, in order
    act = [c for c in range(ncl) if rec["C"][c][1] > 0] if want_few else []
    assert few_ncl == len(act)
    jb = 0
    for k, c in enumerate(act):
        assert rec["F"][k] == [c, rec["C"][c][0], jb]
        jb += int(ns[c])
    assert rec["J"][0] == jb
    work = large_items if want_large else small
    assert (small if want_large else large_items) == 0
    if f32c:
        W = sum((-(-rec["C"][c][1] // cs) if not want_few else 0) * int(njt[c]) for c in range(ncl))
        assert n_units == W and rec["E"][2] == W
        for c in range(ncl):
            assert rec["C"][c][4] == sum((-(-rec["C"][k][1] // cs) if not want_few else 0) * int(njt[k])
                                         for k in range(c))
        workers = p["workers_large"] if want_large else p["workers_small"]
        if chunks == 0:
            assert n_workers == 0 and work == 0
        else:
            assert work == n_workers and 1 <= n_workers <= workers
            assert W // n_workers >= 2 or W < 2        # at least two units a range
            assert n_workers <= p["sms"] or n_workers % p["sms"] == 0
            cap = min(workers, W // 2)
            assert n_workers >= min(cap, p["sms"]) or cap < 1  # rounded down by less than one SM count
    else:
        assert 1 <= split <= p["max_split"] and work == n_items
        items = sum((-(-rec["C"][c][1] // cs)) * min(split, max(int(njt[c]), 1)) for c in range(ncl)) if not want_few else 0
        assert n_items == items and rec["E"][1] == items


@pytest.mark.parametrize("f32c", [True, False])
def test_plan_matches_its_definitions(harness, f32c):
    rng = np.random.default_rng(23 + int(f32c))
    tile, tj = (256, 256) if f32c else (2048, 256)
    for _ in range(120):
        ncl = int(rng.integers(1, 12))
        ns, njt, first = layout(rng, ncl, tile, tj, int(rng.choice([300, 5000, 60000])))
        nu = int(first[-1])
        # sparse, dense or empty activity
        kind = rng.integers(0, 3)
        if kind == 0:
            counts = (rng.random(nu) < 0.02).astype(int)
        elif kind == 1:
            counts = rng.integers(0, 40, nu)
        else:
            counts = np.zeros(nu, dtype=int)
        counts = np.minimum(counts, tile)
        rec = plan(harness, f32c, ns, njt, first, counts)
        check(rec, f32c, ns, njt, first, counts)


def test_plan_at_the_bench_shapes(harness):
    # N = 102 400 in one cluster (400 tiles of 256): one particle, 80, 475,
    # 1700 and all active
    ns, njt, first = np.array([102400]), np.array([400]), np.array([0, 400])
    for n_act in (1, 80, 475, 1719, 102400):
        counts = np.zeros(400, dtype=int)
        idx = np.linspace(0, 102399, n_act).astype(int)
        np.add.at(counts, idx // 256, 1)
        rec = plan(harness, True, ns, njt, first, counts)
        check(rec, True, ns, njt, first, counts)
    rec = plan(harness, True, ns, njt, first, np.bincount(np.arange(80) * 1280 // 256, minlength=400))
    assert rec["S"][9] == 304  # 2 chunks x 400 units over the small kernel's 304 CTAs, two per SM
