"""FP64 CPU oracle of the SCF / MEX expansion force calculation.

TEST INFRASTRUCTURE ONLY.  This package wraps ``etics_oracle.c`` (plain C,
double precision, written from the paper's formulas) with ``ctypes``.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product package never does.  It shares no
code with the CUDA library.

Citations are to the paper's sections and equations (Meiron, Li,
Holley-Bockelmann & Spurzem, "Expansion Techniques for Collisionless Stellar
Dynamical Simulations"):

* ``scf_coeffs`` / ``scf_field``: Sec. 2.4 eq. 18 with the Hernquist-Ostriker
  radial basis of Sec. 2.5 (two passes of Sec. 3.3), or with the
  Clutton-Brock basis Sec. 2.5 names (``basis=CB``).
* ``mex_field``: Sec. 2.4 eqs. 15-17 with the sorted cumulative sums of
  Sec. 2.2 and Sec. 3.2.
* ``direct``: Sec. 2.1 eq. 4.
* ``leapfrog_step``: the kick-drift-kick step mentioned in Secs. 3.4 and 5.4.

``oracle.mlp`` (numpy) is the FP64 oracle of the coefficient-forecasting MLP
and its feature / update glue; the paper has no learned part.

Parity: every function here is pinned by ``tests/test_oracle_*.py`` against
closed forms, quadrature identities, brute force or invariants, and every
function of ``oracle.mlp`` by ``tests/test_oracle_mlp.py`` (none is "parity
unpinned").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "etics_oracle.c")
_LIB = os.path.join(_HERE, "libetics_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (``-O2 -ffp-contract=off``) into the package dir."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB) >= os.path.getmtime(os.path.join(_HERE, "etics_oracle.h"))):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        c_int, c_long, c_double = ctypes.c_int, ctypes.c_long, ctypes.c_double
        lib.etics_ref_phi_nl.argtypes = [c_int, c_int, c_double, dp, dp]
        lib.etics_ref_jnl.argtypes = [c_int, c_int]
        lib.etics_ref_jnl.restype = c_double
        lib.etics_ref_ylm.argtypes = [c_int, c_double, c_double, c_double, dp]
        lib.etics_ref_scf_coeffs.argtypes = [dp, dp, c_long, c_int, c_int, dp]
        lib.etics_ref_scf_field.argtypes = [dp, c_long, c_int, c_int, dp, dp, dp, c_int]
        lib.etics_ref_mex_field.argtypes = [dp, dp, c_long, c_int, dp, dp, lp]
        lib.etics_ref_direct.argtypes = [dp, dp, c_long, dp, dp, c_int]
        lib.etics_ref_leapfrog_step.argtypes = [dp, dp, dp, dp, dp, c_long, c_double,
                                                c_int, c_int, c_int, dp, c_int]
        lib.etics_ref_default_threads.restype = c_int
        lib.etics_ref_phi_nl_b.argtypes = [c_int, c_int, c_int, c_double, dp, dp]
        lib.etics_ref_jnl_b.argtypes = [c_int, c_int, c_int]
        lib.etics_ref_jnl_b.restype = c_double
        lib.etics_ref_scf_coeffs_b.argtypes = [c_int, dp, dp, c_long, c_int, c_int, dp]
        lib.etics_ref_scf_coeffs_bt.argtypes = [c_int, dp, dp, c_long, c_int, c_int, dp, c_int]
        lib.etics_ref_mex_field_t.argtypes = [dp, dp, c_long, c_int, dp, dp, lp, c_int]
        lib.etics_ref_scf_field_b.argtypes = [c_int, dp, c_long, c_int, c_int, dp, dp, dp, c_int]
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pos(pos):
    p = np.ascontiguousarray(pos, dtype=np.float64)
    if p.ndim != 2 or p.shape[1] != 3:
        raise ValueError("positions must have shape (N, 3)")
    return p


def _check(rc, name):
    if rc != 0:
        raise ValueError(f"{name}: bad arguments (status {rc})")


def default_threads() -> int:
    return int(_load().etics_ref_default_threads())


HO, CB = 0, 1     # radial bases of Sec. 2.5: Hernquist-Ostriker, Clutton-Brock


def phi_nl(n: int, l: int, r: float, basis: int = HO):
    """Radial potential basis phi_nl(r) and d phi_nl/dr (Sec. 2.5)."""
    lib = _load()
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib.etics_ref_phi_nl_b(basis, n, l, float(r), ctypes.byref(a), ctypes.byref(b)),
           "phi_nl")
    return a.value, b.value


def jnl(n: int, l: int, basis: int = HO) -> float:
    """Normalisation integral of rho_nl * phi_nl * r^2 (Sec. 2.5 basis)."""
    return float(_load().etics_ref_jnl_b(basis, n, l))


def ylm(l_max: int, x: float, y: float, z: float) -> np.ndarray:
    """Real orthonormal Y_lm (no Condon-Shortley phase), index l*l+l+m."""
    out = np.zeros((l_max + 1) ** 2)
    _check(_load().etics_ref_ylm(l_max, float(x), float(y), float(z), _dp(out)), "ylm")
    return out


def scf_coeffs(pos, mass, n_max: int, l_max: int, basis: int = HO,
               nthreads: int = 0) -> np.ndarray:
    """SCF coefficients c[n, l*l+l+m] (Sec. 2.4 eq. 18), shape (n_max+1, (l_max+1)^2);
    nthreads <= 0 uses every online core (the result is the same for any count)."""
    p = _pos(pos)
    m = np.ascontiguousarray(mass, dtype=np.float64)
    out = np.zeros((n_max + 1, (l_max + 1) ** 2))
    _check(_load().etics_ref_scf_coeffs_bt(basis, _dp(p), _dp(m), len(p), n_max, l_max,
                                           _dp(out), int(nthreads)), "scf_coeffs")
    return out


def scf_field(pos, n_max: int, l_max: int, coeffs, nthreads: int = 0, basis: int = HO):
    """SCF acceleration (N,3) and potential (N,) at arbitrary points."""
    p = _pos(pos)
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    if c.shape != (n_max + 1, (l_max + 1) ** 2):
        raise ValueError("coefficient shape mismatch")
    acc = np.zeros((len(p), 3))
    pot = np.zeros(len(p))
    _check(_load().etics_ref_scf_field_b(basis, _dp(p), len(p), n_max, l_max, _dp(c),
                                         _dp(acc), _dp(pot), int(nthreads)), "scf_field")
    return acc, pot


def mex_field(pos, mass, l_max: int, nthreads: int = 0):
    """MEX acceleration, potential and the radial order (Sec. 2.4 eqs. 15-17);
    nthreads <= 0 uses every online core (the result is the same for any count)."""
    p = _pos(pos)
    m = np.ascontiguousarray(mass, dtype=np.float64)
    acc = np.zeros((len(p), 3))
    pot = np.zeros(len(p))
    order = np.zeros(len(p), dtype=np.int64)
    _check(_load().etics_ref_mex_field_t(_dp(p), _dp(m), len(p), l_max, _dp(acc), _dp(pot),
                                         order.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                         int(nthreads)),
           "mex_field")
    return acc, pot, order


def direct(pos, mass, nthreads: int = 0):
    """Unsoftened direct summation (Sec. 2.1 eq. 4), self term excluded."""
    p = _pos(pos)
    m = np.ascontiguousarray(mass, dtype=np.float64)
    acc = np.zeros((len(p), 3))
    pot = np.zeros(len(p))
    _check(_load().etics_ref_direct(_dp(p), _dp(m), len(p), _dp(acc), _dp(pot), int(nthreads)),
           "direct")
    return acc, pot


def leapfrog_step(pos, vel, mass, acc, dt: float, method: int, n_max: int, l_max: int,
                  nthreads: int = 0):
    """One KDK step in place on (pos, vel, acc); returns (pot, coeffs or None)."""
    for a in (pos, vel, acc):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("pos, vel, acc must be C-contiguous float64 arrays")
    m = np.ascontiguousarray(mass, dtype=np.float64)
    pot = np.zeros(len(pos))
    coeffs = np.zeros((n_max + 1, (l_max + 1) ** 2)) if method == 0 else None
    _check(_load().etics_ref_leapfrog_step(
        _dp(pos), _dp(vel), _dp(m), _dp(acc), _dp(pot), len(pos), float(dt), int(method),
        int(n_max), int(l_max), _dp(coeffs) if coeffs is not None else None, int(nthreads)),
        "leapfrog_step")
    return pot, coeffs
