"""Plain FP64 CPU oracle for direct-summation gravity (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library and its Python binding
never call it; it shares no code with them.

The arithmetic lives in ``nbody_oracle.c`` (compiled with ``gcc -O2 -fopenmp``,
no fast-math).  This module only builds it and marshals numpy arrays:

* ``forces``       -- a_i and phi_i for every i (Sec. 3 force sum, divided by m_i,
  with Plummer softening; j = i excluded).
* ``forces_rows``  -- the same for a chosen subset of rows (for sampled checks at
  large N).
* ``kdk``          -- kick-drift-kick leapfrog in FP64 (the paper keeps the
  integration in double precision on the host, Sec. 3).
* ``energy``       -- K, W, E, P, L.
* ``forces_jerk``  -- a_i, its time derivative (jerk) and phi_i, which the paper
  computes together (Sec. 3); ``forces_jerk_rows`` for a subset of rows.
* ``hermite``      -- the fourth-order Hermite predictor-corrector integrator
  that uses the jerk (shared time step).
* ``block_hermite`` -- the same scheme with individual power-of-two block time
  steps chosen by Aarseth's criterion; ``aarseth_step`` evaluates that criterion
  alone from the acceleration and jerk at both ends of one step.

Layouts follow the C ABI: positions/velocities/accelerations are ``[3, n]``
float64 arrays, masses and potentials ``[n]``.

Parity status: every function here is pinned: the forces, KDK and energies by
``tests/test_oracle_pins.py`` (closed forms, invariants, Kepler orbits,
Plummer virial ratio, the potential-gradient relation), the jerk and shared-step
Hermite by ``tests/test_oracle_jerk_pins.py`` (two-body closed forms, the time
derivative of the acceleration, fourth-order convergence), and the block steps
with their step criterion by ``tests/test_oracle_block_pins.py`` (reduction to
shared steps, a criterion exact for a cubic acceleration history, circular-binary
first and settled steps, convergence); ``tests/test_oracle_mutants.py`` shows
that 24 planted mistakes each fail a pin.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbody_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_default = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile an oracle source into a shared library (gcc, OpenMP, no fast-math)."""
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _c(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """Numpy front end of one compiled oracle library."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        d = ctypes.c_double
        i64 = ctypes.c_int64
        vp = ctypes.c_void_p
        lib.oracle_forces.argtypes = [i64, vp, vp, d, d, vp, vp]
        lib.oracle_forces.restype = None
        lib.oracle_forces_rows.argtypes = [i64, vp, vp, d, d, vp, i64, vp, vp]
        lib.oracle_forces_rows.restype = None
        lib.oracle_energy.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.oracle_energy.restype = None
        lib.oracle_kdk.argtypes = [i64, vp, vp, vp, d, d, d, i64, vp, vp, ctypes.c_int, vp]
        lib.oracle_kdk.restype = None
        lib.oracle_forces_jerk.argtypes = [i64, vp, vp, vp, d, d, vp, vp, vp]
        lib.oracle_forces_jerk.restype = None
        lib.oracle_forces_jerk_rows.argtypes = [i64, vp, vp, vp, d, d, vp, i64, vp, vp, vp]
        lib.oracle_forces_jerk_rows.restype = None
        lib.oracle_hermite.argtypes = [i64, vp, vp, vp, d, d, d, i64, vp, vp, vp, ctypes.c_int, vp]
        lib.oracle_hermite.restype = None
        lib.oracle_block_hermite.argtypes = [i64, vp, vp, vp, d, d, d, d, d, d, d, vp, vp, vp, vp,
                                             ctypes.POINTER(i64)]
        lib.oracle_block_hermite.restype = i64
        lib.oracle_aarseth_step.argtypes = [vp, vp, vp, vp, d, d, d]
        lib.oracle_aarseth_step.restype = d
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    def num_threads(self) -> int:
        return int(self.lib.oracle_num_threads())

    def forces(self, pos, mass, eps: float, G: float = 1.0):
        """Return (acc[3, n], pot[n]) in FP64 for every particle."""
        mass = _c(mass)
        n = mass.shape[0]
        pos = _c(pos, (3, n))
        acc = np.empty((3, n), np.float64)
        pot = np.empty(n, np.float64)
        self.lib.oracle_forces(n, _p(pos), _p(mass), float(eps), float(G), _p(acc), _p(pot))
        return acc, pot

    def forces_rows(self, pos, mass, eps: float, rows, G: float = 1.0):
        """Return (acc[3, k], pot[k]) for the particles listed in ``rows``."""
        mass = _c(mass)
        n = mass.shape[0]
        pos = _c(pos, (3, n))
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        if rows.size and (rows.min() < 0 or rows.max() >= n):
            raise IndexError("row index out of range")
        k = rows.shape[0]
        acc = np.empty((3, k), np.float64)
        pot = np.empty(k, np.float64)
        self.lib.oracle_forces_rows(n, _p(pos), _p(mass), float(eps), float(G), _p(rows), k,
                                    _p(acc), _p(pot))
        return acc, pot

    def energy(self, pos, vel, mass, pot):
        """Return [K, W, E, Px, Py, Pz, Lx, Ly, Lz]."""
        mass = _c(mass)
        n = mass.shape[0]
        pos = _c(pos, (3, n))
        vel = _c(vel, (3, n))
        pot = _c(pot, (n,))
        out = np.empty(9, np.float64)
        self.lib.oracle_energy(n, _p(pos), _p(vel), _p(mass), _p(pot), _p(out))
        return out

    def kdk(self, pos, vel, mass, eps: float, dt: float, nsteps: int, G: float = 1.0, acc=None,
            pot=None, diag: bool = False):
        """Advance copies of (pos, vel) by ``nsteps`` KDK steps.

        Returns (pos, vel, acc, pot, diag) where diag is [nsteps + 1, 9] (row 0
        the initial state) or None.
        """
        mass = _c(mass)
        n = mass.shape[0]
        pos = _c(pos, (3, n)).copy()
        vel = _c(vel, (3, n)).copy()
        have = acc is not None and pot is not None
        acc = _c(acc, (3, n)).copy() if have else np.empty((3, n), np.float64)
        pot = _c(pot, (n,)).copy() if have else np.empty(n, np.float64)
        dg = np.empty((nsteps + 1, 9), np.float64) if diag else None
        self.lib.oracle_kdk(n, _p(pos), _p(vel), _p(mass), float(eps), float(G), float(dt),
                            int(nsteps), _p(acc), _p(pot), int(have),
                            _p(dg) if dg is not None else None)
        return pos, vel, acc, pot, dg


def _forces_jerk(self, pos, vel, mass, eps: float, G: float = 1.0):
    """Return (acc[3, n], jerk[3, n], pot[n]) in FP64."""
    mass = _c(mass)
    n = mass.shape[0]
    pos = _c(pos, (3, n))
    vel = _c(vel, (3, n))
    acc = np.empty((3, n), np.float64)
    jerk = np.empty((3, n), np.float64)
    pot = np.empty(n, np.float64)
    self.lib.oracle_forces_jerk(n, _p(pos), _p(vel), _p(mass), float(eps), float(G), _p(acc),
                                _p(jerk), _p(pot))
    return acc, jerk, pot


def _forces_jerk_rows(self, pos, vel, mass, eps: float, rows, G: float = 1.0):
    """Return (acc[3, k], jerk[3, k], pot[k]) in FP64 for the given rows."""
    mass = _c(mass)
    n = mass.shape[0]
    pos = _c(pos, (3, n))
    vel = _c(vel, (3, n))
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    k = rows.shape[0]
    acc = np.empty((3, k), np.float64)
    jerk = np.empty((3, k), np.float64)
    pot = np.empty(k, np.float64)
    self.lib.oracle_forces_jerk_rows(n, _p(pos), _p(vel), _p(mass), float(eps), float(G), _p(rows), k,
                                     _p(acc), _p(jerk), _p(pot))
    return acc, jerk, pot


def _hermite(self, pos, vel, mass, eps: float, dt: float, nsteps: int, G: float = 1.0,
             diag: bool = False):
    """Advance copies of (pos, vel) by ``nsteps`` Hermite steps.

    Returns (pos, vel, acc, jerk, pot, diag[nsteps + 1, 9] or None).
    """
    mass = _c(mass)
    n = mass.shape[0]
    pos = _c(pos, (3, n)).copy()
    vel = _c(vel, (3, n)).copy()
    acc = np.empty((3, n), np.float64)
    jerk = np.empty((3, n), np.float64)
    pot = np.empty(n, np.float64)
    dg = np.empty((nsteps + 1, 9), np.float64) if diag else None
    self.lib.oracle_hermite(n, _p(pos), _p(vel), _p(mass), float(eps), float(G), float(dt),
                            int(nsteps), _p(acc), _p(jerk), _p(pot), 0,
                            _p(dg) if dg is not None else None)
    return pos, vel, acc, jerk, pot, dg


def _block_hermite(self, pos, vel, mass, eps: float, t_end: float, dt_max: float, dt_min: float,
                   eta: float, eta_s: float, G: float = 1.0):
    """Block-step Hermite to t_end.  Returns (pos, vel, acc, jerk, pot, dt, blocks, evals)."""
    mass = _c(mass)
    n = mass.shape[0]
    pos = _c(pos, (3, n)).copy()
    vel = _c(vel, (3, n)).copy()
    acc = np.empty((3, n), np.float64)
    jerk = np.empty((3, n), np.float64)
    pot = np.empty(n, np.float64)
    dt = np.empty(n, np.float64)
    ev = ctypes.c_int64()
    blocks = self.lib.oracle_block_hermite(n, _p(pos), _p(vel), _p(mass), float(eps), float(G),
                                           float(t_end), float(dt_max), float(dt_min), float(eta),
                                           float(eta_s), _p(acc), _p(jerk), _p(pot), _p(dt),
                                           ctypes.byref(ev))
    return pos, vel, acc, jerk, pot, dt, int(blocks), int(ev.value)


def _aarseth_step(self, a0, j0, a1, j1, h: float, eta: float, dt_max: float = float("inf")):
    """Aarseth's step criterion from the acceleration and jerk at both ends of a
    step of length h (the block integrator's next-step rule, before rounding to
    a power of two)."""
    v = [_c(x, (3,)) for x in (a0, j0, a1, j1)]
    return float(self.lib.oracle_aarseth_step(*[_p(x) for x in v], float(h), float(eta),
                                              float(dt_max)))


Oracle.aarseth_step = _aarseth_step
Oracle.block_hermite = _block_hermite
Oracle.forces_jerk = _forces_jerk
Oracle.forces_jerk_rows = _forces_jerk_rows
Oracle.hermite = _hermite


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def num_threads() -> int:
    return default().num_threads()


def forces(pos, mass, eps: float, G: float = 1.0):
    return default().forces(pos, mass, eps, G)


def forces_rows(pos, mass, eps: float, rows, G: float = 1.0):
    return default().forces_rows(pos, mass, eps, rows, G)


def energy(pos, vel, mass, pot):
    return default().energy(pos, vel, mass, pot)


def kdk(pos, vel, mass, eps: float, dt: float, nsteps: int, G: float = 1.0, acc=None, pot=None,
        diag: bool = False):
    return default().kdk(pos, vel, mass, eps, dt, nsteps, G, acc, pot, diag)
