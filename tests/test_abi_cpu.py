"""The C ABI library loads and exports every entry point of include/nbody.h (CPU only).

No compute call is made here (there may be no GPU); only host-side behaviour
is checked: symbol export, status strings, the table of compiled tile shapes
and argument validation that happens before any device work.
"""
import ctypes
import os
import re

import pytest

import paper_2509_19294_gb300 as nb
from paper_2509_19294_gb300 import build as nbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    nbuild.build()
    return nb.load()


def _header_functions():
    text = open(os.path.join(ROOT, "include", "nbody.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nbody_[a-z_]+)\s*\(", text)))


def test_header_declares_the_four_core_calls():
    names = _header_functions()
    for core in ("nbody_init", "nbody_forces", "nbody_step", "nbody_energy"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    names = _header_functions()
    assert names, "no declarations parsed"
    for name in names:
        assert hasattr(lib, name), f"{name} declared in nbody.h but not exported"
    assert set(names) == set(nb.EXPORTED)


def test_probe_library_is_separate_from_the_force_library(lib):
    # the benchmark's pipe-rate probe lives in libnbody_probe.so with its own
    # header; the force library's ABI does not carry it
    from paper_2509_19294_gb300 import probe
    plib = probe.load()
    assert hasattr(plib, "nbody_measure_pipes")
    text = open(os.path.join(ROOT, "paper_2509_19294_gb300", "probe", "pipe_rates.h")).read()
    assert "int nbody_measure_pipes(double *out, int n_out);" in text
    assert "nbody_measure_pipes" not in _header_functions()
    with pytest.raises(AttributeError):
        getattr(lib, "nbody_measure_pipes")


def test_status_strings(lib):
    assert nb.nbody_strerror(0) == "success"
    assert "invalid" in nb.nbody_strerror(nb.NBODY_EINVAL)
    assert nb.nbody_strerror(12345) == "unknown status"


def test_tile_table_is_consistent(lib):
    shapes = nb.nbody_tiles_supported()
    assert len(shapes) >= 4
    for block, p, tj, minb in shapes:
        assert block % 32 == 0 and tj % 8 == 0 and (block * p) % tj == 0 and minb >= 1


def test_init_rejects_bad_configs_before_touching_the_device(lib):
    bad = [
        dict(n_total=-1, eps=0.1),
        dict(n_total=10, eps=-0.1),
        dict(n_total=10, eps=float("nan")),
        dict(n_total=10, eps=0.1, G=float("inf")),
        dict(n_total=10, eps=0.1, mode=7),
        dict(n_total=10, eps=[0.1, 0.1], cluster_offsets=[0, 6, 5]),
        dict(n_total=10, eps=[0.1, 0.1], cluster_offsets=[0, 4, 9]),
        dict(n_total=10, eps=0.1, reorder_every=-2),
    ]
    for kw in bad:
        with pytest.raises(nb.NBodyError) as e:
            nb.nbody_init(**kw)
        assert e.value.code == nb.NBODY_EINVAL, kw


def test_calls_on_null_context_fail_cleanly(lib):
    assert lib.nbody_forces(None, None, None, None, None, None) == nb.NBODY_EINVAL
    assert lib.nbody_get_tiles(None, None) == nb.NBODY_EINVAL
    assert lib.nbody_kernel_launches(None) == 0
    lib.nbody_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path):
    import importlib
    mod = importlib.reload(nb)
    try:
        mod._lib = None
        with pytest.raises(RuntimeError, match="missing"):
            mod.load(str(tmp_path / "absent.so"))
    finally:
        importlib.reload(nb)
