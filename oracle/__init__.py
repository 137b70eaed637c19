"""CPU oracle for checkerboard-overrelaxation SU(3) gauge fixing (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline leg of
the benchmark may import this package; the CUDA product path never does.  It wraps
``gf_oracle.c`` (plain FP64 C, one site at a time, Section 1 Eqs. (1)-(6) and
Algorithm 1 of the paper) through ctypes.  Arrays are canonical complex128 fields of
shape (Lt, Lz, Ly, Lx, 4, 3, 3); every function works in place or returns new numpy
arrays and never touches a GPU.

Parity status of each function (what pins it) is listed in the test files
``tests/test_oracle_*.py``; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libgf_oracle.so")
_lock = threading.Lock()
_lib = None

LANDAU, COULOMB = 0, 1
OR_FIRST_ORDER, OR_EXACT = 0, 1

_CP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source file with gcc (FP64, no FMA contraction, OpenMP)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile gf_oracle.c into oracle/_build/libgf_oracle.so if it is missing or stale."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        return compile_source(_SRC, _LIB)


def _bind(path: str):
    lib = ctypes.CDLL(path)
    lib.orc_measure.argtypes = [_CP, _IP, ctypes.c_int, _DP, _DP, _DP, _DP]
    lib.orc_delta.argtypes = [_CP, _IP, ctypes.c_int, _CP]
    lib.orc_su2_maximiser.argtypes = [_CP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_int, _CP, _CP]
    lib.orc_su2_maximiser.restype = None
    lib.orc_or_half_sweep.argtypes = [_CP, _IP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, _CP]
    lib.orc_reunit.argtypes = [_CP, ctypes.c_long]
    lib.orc_reunit.restype = None
    lib.orc_fix.argtypes = [_CP, _IP, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                            ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            _IP, _DP, _DP, _DP, _IP]
    lib.orc_num_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


class _Variant:
    """The same API bound to another build of the oracle (used to plant mistakes in tests)."""

    def __init__(self, path: str):
        self._lib = _bind(path)

    def __getattr__(self, name):
        fn = globals()[name]
        if not callable(fn):
            return fn

        def call(*args, **kw):
            global _lib
            saved = _lib
            _lib = self._lib
            try:
                return fn(*args, **kw)
            finally:
                _lib = saved
        return call


def load_variant(path: str) -> "_Variant":
    return _Variant(path)


def _dims_of(U: np.ndarray):
    if U.dtype != np.complex128 or U.ndim != 7 or U.shape[4:] != (4, 3, 3):
        raise ValueError("expected a complex128 field of shape (Lt, Lz, Ly, Lx, 4, 3, 3)")
    if not U.flags.c_contiguous:
        raise ValueError("field must be C-contiguous")
    Lt, Lz, Ly, Lx = U.shape[:4]
    return (ctypes.c_int * 4)(Lx, Ly, Lz, Lt)


def _nd(gauge: int) -> int:
    return 4 if gauge == LANDAU else 3


def num_threads() -> int:
    return int(_load().orc_num_threads())


def measure(U: np.ndarray, gauge: int = LANDAU):
    """(F, theta, F_t, theta_t) by Eqs. (1)-(3); per-slice arrays have Lt entries."""
    lib = _load()
    L = _dims_of(U)
    Lt = U.shape[0]
    F, th = ctypes.c_double(), ctypes.c_double()
    F_t, th_t = np.zeros(Lt), np.zeros(Lt)
    rc = lib.orc_measure(U.ctypes.data, L, _nd(gauge), ctypes.byref(F), ctypes.byref(th),
                         F_t.ctypes.data_as(_DP), th_t.ctypes.data_as(_DP))
    if rc != 0:
        raise ValueError(f"orc_measure failed ({rc})")
    return F.value, th.value, F_t, th_t


def delta(U: np.ndarray, gauge: int = LANDAU) -> np.ndarray:
    """Delta(x) of Eq. (3) at every site, shape (Lt, Lz, Ly, Lx, 3, 3)."""
    lib = _load()
    L = _dims_of(U)
    out = np.zeros(U.shape[:4] + (3, 3), dtype=np.complex128)
    if lib.orc_delta(U.ctypes.data, L, _nd(gauge), out.ctypes.data) != 0:
        raise ValueError("orc_delta failed")
    return out


def su2_maximiser(K: np.ndarray, i: int, j: int, omega: float = 1.0, form: int = OR_FIRST_ORDER):
    """(a, b) of the subgroup element maximising Re Tr[R K] on rows (i, j), then R^omega."""
    lib = _load()
    K = np.ascontiguousarray(K, dtype=np.complex128)
    a = np.zeros(1, np.complex128)
    b = np.zeros(1, np.complex128)
    lib.orc_su2_maximiser(K.ctypes.data, i, j, omega, form, a.ctypes.data, b.ctypes.data)
    return complex(a[0]), complex(b[0])


def or_half_sweep(U: np.ndarray, parity: int, omega: float = 1.7, gauge: int = LANDAU,
                  form: int = OR_FIRST_ORDER, reunit_after: bool = False, slice_active=None):
    """One checkerboard half-sweep of Algorithm 1, in place."""
    lib = _load()
    L = _dims_of(U)
    mask = None
    if slice_active is not None:
        mask = np.ascontiguousarray(slice_active, dtype=np.uint8)
        if mask.shape != (U.shape[0],):
            raise ValueError("slice_active must have Lt entries")
    rc = lib.orc_or_half_sweep(U.ctypes.data, L, _nd(gauge), parity, omega, form,
                               int(bool(reunit_after)), None if mask is None else mask.ctypes.data)
    if rc != 0:
        raise ValueError(f"orc_or_half_sweep failed ({rc})")
    return U


def sweep(U: np.ndarray, omega: float = 1.7, gauge: int = LANDAU, form: int = OR_FIRST_ORDER,
          reunit: bool = False):
    """Even then odd half-sweep; `reunit` reunitarises after the odd half-sweep."""
    or_half_sweep(U, 0, omega, gauge, form, False)
    or_half_sweep(U, 1, omega, gauge, form, reunit)
    return U


def reunit(U: np.ndarray) -> np.ndarray:
    lib = _load()
    if U.dtype != np.complex128 or not U.flags.c_contiguous or U.shape[-2:] != (3, 3):
        raise ValueError("expected a C-contiguous complex128 array of 3x3 matrices")
    lib.orc_reunit(U.ctypes.data, U.size // 9)
    return U


def fix(U: np.ndarray, eps: float, maxiter: int, omega: float = 1.7, gauge: int = LANDAU,
        form: int = OR_FIRST_ORDER, reunit_interval: int = 20, per_slice: bool | None = None):
    """Algorithm 1 in place.  Returns dict(rc, iters, F, theta, theta_hist, slice_iters).

    rc = 0 converged, 1 maxiter reached.  per_slice defaults to True for Coulomb gauge.
    """
    lib = _load()
    L = _dims_of(U)
    if per_slice is None:
        per_slice = gauge == COULOMB
    it = ctypes.c_int()
    F, th = ctypes.c_double(), ctypes.c_double()
    hist = np.full(maxiter + 1, np.nan)
    sl = np.zeros(U.shape[0], dtype=np.int32)
    rc = lib.orc_fix(U.ctypes.data, L, _nd(gauge), omega, form, eps, maxiter, reunit_interval,
                     int(bool(per_slice)), ctypes.byref(it), ctypes.byref(F), ctypes.byref(th),
                     hist.ctypes.data_as(_DP), sl.ctypes.data_as(_IP))
    if rc < 0:
        raise ValueError(f"orc_fix failed ({rc})")
    return dict(rc=rc, iters=it.value, F=F.value, theta=th.value,
                theta_hist=hist[: it.value + 1], slice_iters=sl)
