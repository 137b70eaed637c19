"""Thin Python binding of libgf (the C ABI in include/gf.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does nothing but
convert arguments, call it and raise GFError on a negative status.  All computation
runs in the CUDA library; importing this module fails loudly when the library has not
been built (there is no CPU fallback).

``GaugeFixer`` is a convenience owner of a handle whose device workspace is a torch
tensor (torch's caching allocator supplies the memory) and whose stream is torch's
current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgf.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "gf.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)

# constants of include/gf.h
GF_OK, GF_ENOTCONVERGED, GF_EINVAL, GF_ECUDA, GF_ENOMEM, GF_ESTATE = 0, 1, -1, -2, -3, -4
GF_LANDAU, GF_COULOMB = 0, 1
GF_FP64_18, GF_FP32_18, GF_FP32_12, GF_FP64_12, GF_FP32_8, GF_FP64_8 = 0, 1, 2, 3, 4, 5
GF_FLAG_MIXED = 1
GF_FLAG_FASD = 2
GF_FLAG_AUTOGRAD = 4
GF_METHOD_OR, GF_METHOD_FASD = 0, 1
GF_OR_FIRST_ORDER, GF_OR_EXACT = 0, 1
GF_SWEEP_AUTO, GF_SWEEP_REGISTER, GF_SWEEP_PIPELINED = 0, 1, 2
GF_POLISH_FP64, GF_POLISH_SPLIT = 0, 1

_vp, _int, _dbl, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
_IP, _DP = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "gf_workspace_bytes": (_int, [_int, _IP, _int, _int, _int, ctypes.POINTER(_sz)]),
    "gf_create": (_int, [_IP, _int, _int, _int, _int, _vp, _vp, _sz, ctypes.POINTER(_vp)]),
    "gf_create_batch": (_int, [_int, _IP, _int, _int, _int, _vp, _vp, _sz, ctypes.POINTER(_vp)]),
    "gf_destroy": (None, [_vp]),
    "gf_last_error": (ctypes.c_char_p, [_vp]),
    "gf_num_lattices": (_int, [_vp]),
    "gf_num_units": (_int, [_vp]),
    "gf_upload": (_int, [_vp, _int, _vp, _int]),
    "gf_download": (_int, [_vp, _int, _vp, _int]),
    "gf_functional_theta": (_int, [_vp, _DP, _DP, _DP, _DP]),
    "gf_or_sweep": (_int, [_vp, _int, _dbl]),
    "gf_reunitarize": (_int, [_vp]),
    "gf_fix": (_int, [_vp, _dbl, _int, _IP, _DP, _DP]),
    "gf_set_omega": (_int, [_vp, _dbl]),
    "gf_set_overrelax_form": (_int, [_vp, _int]),
    "gf_set_reunit_interval": (_int, [_vp, _int]),
    "gf_set_check_interval": (_int, [_vp, _int]),
    "gf_set_mixed_switch": (_int, [_vp, _dbl]),
    "gf_set_reproducible": (_int, [_vp, _int]),
    "gf_set_block_size": (_int, [_vp, _int]),
    "gf_fix_phase_sweeps": (_int, [_vp, _IP, _IP]),
    "gf_set_sweep_variant": (_int, [_vp, _int]),
    "gf_set_polish": (_int, [_vp, _int]),
    "gf_autotune": (_int, [_vp, _IP, _IP]),
    "gf_get_sweeps_done": (_int, [_vp, _IP]),
    "gf_set_sweeps_done": (_int, [_vp, _int]),
    "gf_set_history": (_int, [_vp, _vp, _int]),
    "gf_history_count": (_int, [_vp, _IP]),
    "gf_fa_sd_step": (_int, [_vp, _dbl]),
    "gf_set_method": (_int, [_vp, _int]),
    "gf_set_alpha": (_int, [_vp, _dbl]),
    "gf_ad_functional": (_int, [_vp, _vp, _vp]),
    "gf_ad_backward": (_int, [_vp, _vp, _vp, _vp]),
    "gf_functional_theta_noalloc": (_int, [_IP, _int, _vp, _vp, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def header_symbols() -> list[str]:
    """Entry points declared in include/gf.h."""
    return re.findall(r"^GF_API[^(]*?\b(gf_\w+)\s*\(", open(HEADER).read(), flags=re.M)


class GFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libgf error {code}: {msg}")
        self.code = code


def _check(rc: int, h=None) -> int:
    if rc < 0:
        raise GFError(rc, gf_last_error(h))
    return rc


def _dims_array(dims) -> "ctypes.Array":
    flat = [int(v) for d in dims for v in d]
    return (ctypes.c_int * len(flat))(*flat)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def gf_last_error(h=None) -> str:
    s = _lib.gf_last_error(h)
    return s.decode() if s else ""


def gf_workspace_bytes(dims_list, gauge: int, storage: int, flags: int = 0) -> int:
    out = _sz()
    _check(_lib.gf_workspace_bytes(len(dims_list), _dims_array(dims_list), gauge, storage, flags,
                                   ctypes.byref(out)))
    return out.value


def gf_create(dims, nc: int, gauge: int, storage: int, flags: int = 0, stream: int = 0,
              workspace: int = 0, workspace_bytes: int = 0):
    h = _vp()
    _check(_lib.gf_create((ctypes.c_int * 4)(*[int(v) for v in dims]), nc, gauge, storage, flags,
                          _vp(stream or None), _vp(workspace or None), workspace_bytes, ctypes.byref(h)))
    return h


def gf_create_batch(dims_list, gauge: int, storage: int, flags: int = 0, stream: int = 0,
                    workspace: int = 0, workspace_bytes: int = 0):
    h = _vp()
    _check(_lib.gf_create_batch(len(dims_list), _dims_array(dims_list), gauge, storage, flags,
                                _vp(stream or None), _vp(workspace or None), workspace_bytes,
                                ctypes.byref(h)))
    return h


def gf_destroy(h) -> None:
    _lib.gf_destroy(h)


def gf_num_lattices(h) -> int:
    return _check(_lib.gf_num_lattices(h), h)


def gf_num_units(h) -> int:
    return _check(_lib.gf_num_units(h), h)


def gf_upload(h, lat: int, ptr: int, on_device: bool) -> None:
    _check(_lib.gf_upload(h, lat, _vp(ptr), int(on_device)), h)


def gf_download(h, lat: int, ptr: int, on_device: bool) -> None:
    _check(_lib.gf_download(h, lat, _vp(ptr), int(on_device)), h)


def gf_functional_theta(h):
    """(F[n_lat], theta[n_lat], unit_F[n_units], unit_theta[n_units])."""
    nl, nu = gf_num_lattices(h), gf_num_units(h)
    F, th, uF, uT = np.zeros(nl), np.zeros(nl), np.zeros(nu), np.zeros(nu)
    _check(_lib.gf_functional_theta(h, _dptr(F), _dptr(th), _dptr(uF), _dptr(uT)), h)
    return F, th, uF, uT


def gf_or_sweep(h, parity: int, omega: float) -> None:
    _check(_lib.gf_or_sweep(h, parity, omega), h)


def gf_reunitarize(h) -> None:
    _check(_lib.gf_reunitarize(h), h)


def gf_fix(h, eps: float, maxiter: int):
    """(status, iters[n_units], F[n_lat], theta[n_lat]); status GF_OK or GF_ENOTCONVERGED."""
    nl, nu = gf_num_lattices(h), gf_num_units(h)
    it = np.zeros(nu, dtype=np.int32)
    F, th = np.zeros(nl), np.zeros(nl)
    rc = _check(_lib.gf_fix(h, eps, maxiter, it.ctypes.data_as(_IP), _dptr(F), _dptr(th)), h)
    return rc, it, F, th


def gf_set_omega(h, omega: float) -> None:
    _check(_lib.gf_set_omega(h, omega), h)


def gf_set_overrelax_form(h, form: int) -> None:
    _check(_lib.gf_set_overrelax_form(h, form), h)


def gf_set_reunit_interval(h, n: int) -> None:
    _check(_lib.gf_set_reunit_interval(h, n), h)


def gf_set_check_interval(h, n: int) -> None:
    _check(_lib.gf_set_check_interval(h, n), h)


def gf_set_mixed_switch(h, eps_sw: float) -> None:
    _check(_lib.gf_set_mixed_switch(h, eps_sw), h)


def gf_set_reproducible(h, on: bool) -> None:
    _check(_lib.gf_set_reproducible(h, int(bool(on))), h)


def gf_set_block_size(h, threads: int) -> None:
    _check(_lib.gf_set_block_size(h, threads), h)


def gf_fa_sd_step(h, alpha: float = 0.08) -> None:
    _check(_lib.gf_fa_sd_step(h, alpha), h)


def gf_set_method(h, method: int) -> None:
    _check(_lib.gf_set_method(h, method), h)


def gf_set_alpha(h, alpha: float) -> None:
    _check(_lib.gf_set_alpha(h, alpha), h)


def gf_ad_functional(h, c_ptr: int, out_ptr: int) -> None:
    _check(_lib.gf_ad_functional(h, _vp(c_ptr or None), _vp(out_ptr or None)), h)


def gf_ad_backward(h, c_ptr: int, upstream_ptr: int, grad_ptr: int) -> None:
    _check(_lib.gf_ad_backward(h, _vp(c_ptr or None), _vp(upstream_ptr or None), _vp(grad_ptr or None)), h)


def gf_set_polish(h, polish: int) -> None:
    _check(_lib.gf_set_polish(h, polish), h)


def gf_set_sweep_variant(h, variant: int) -> None:
    _check(_lib.gf_set_sweep_variant(h, variant), h)


def gf_autotune(h):
    """(threads, variant) picked by the library's autotuner."""
    t, v = ctypes.c_int(), ctypes.c_int()
    _check(_lib.gf_autotune(h, ctypes.byref(t), ctypes.byref(v)), h)
    return t.value, v.value


def gf_get_sweeps_done(h) -> int:
    n = ctypes.c_int()
    _check(_lib.gf_get_sweeps_done(h, ctypes.byref(n)), h)
    return n.value


def gf_set_sweeps_done(h, n: int) -> None:
    _check(_lib.gf_set_sweeps_done(h, n), h)


def gf_set_history(h, buf_ptr: int, capacity: int) -> None:
    _check(_lib.gf_set_history(h, ctypes.c_void_p(buf_ptr), capacity), h)


def gf_history_count(h) -> int:
    n = ctypes.c_int()
    _check(_lib.gf_history_count(h, ctypes.byref(n)), h)
    return n.value


def gf_fix_phase_sweeps(h):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(_lib.gf_fix_phase_sweeps(h, ctypes.byref(a), ctypes.byref(b)), h)
    return a.value, b.value


def gf_functional_theta_noalloc(dims, gauge: int, links_ptr: int, out_ptr: int, stream: int = 0) -> None:
    """F, theta of a canonical device field into out_ptr[0:2] (device), no allocation."""
    _check(_lib.gf_functional_theta_noalloc((ctypes.c_int * 4)(*[int(v) for v in dims]), gauge,
                                            _vp(links_ptr or None), _vp(out_ptr or None), _vp(stream or None)))


# ------------------------------------------------------------------------------------
# Convenience owner: torch supplies the device workspace and the stream
# ------------------------------------------------------------------------------------
def _canonical_ptr(U, dims):
    """(pointer, on_device, keepalive) of a canonical complex128 field (numpy or torch)."""
    Lx, Ly, Lz, Lt = dims
    shape = (Lt, Lz, Ly, Lx, 4, 3, 3)
    if isinstance(U, np.ndarray):
        if U.dtype != np.complex128 or tuple(U.shape) != shape or not U.flags.c_contiguous:
            raise ValueError(f"expected a C-contiguous complex128 array of shape {shape}")
        return U.ctypes.data, False, U
    import torch
    if U.dtype != torch.complex128 or tuple(U.shape) != shape or not U.is_contiguous():
        raise ValueError(f"expected a contiguous complex128 tensor of shape {shape}")
    return U.data_ptr(), U.is_cuda, U


class GaugeFixer:
    """One handle over one lattice or a batch; memory and stream from torch."""

    def __init__(self, dims, gauge: int = GF_LANDAU, storage: int = GF_FP32_12, mixed: bool = False,
                 device=None, stream=None, fasd: bool = False, autograd: bool = False):
        import torch
        self.dims_list = [tuple(int(v) for v in d) for d in (dims if isinstance(dims[0], (list, tuple)) else [dims])]
        self.device = torch.device(device if device is not None else "cuda")
        flags = ((GF_FLAG_MIXED if mixed else 0) | (GF_FLAG_FASD if fasd else 0)
                 | (GF_FLAG_AUTOGRAD if autograd else 0))
        nbytes = gf_workspace_bytes(self.dims_list, gauge, storage, flags)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h = gf_create_batch(self.dims_list, gauge, storage, flags, self.stream.cuda_stream,
                                 self.workspace.data_ptr(), nbytes)
        self.gauge, self.storage = gauge, storage

    def close(self):
        if getattr(self, "h", None):
            gf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload(self, U, lat: int = 0):
        ptr, dev, _keep = _canonical_ptr(U, self.dims_list[lat])
        gf_upload(self.h, lat, ptr, dev)

    def download(self, lat: int = 0, out=None):
        Lx, Ly, Lz, Lt = self.dims_list[lat]
        if out is None:
            out = np.empty((Lt, Lz, Ly, Lx, 4, 3, 3), dtype=np.complex128)
        ptr, dev, _keep = _canonical_ptr(out, self.dims_list[lat])
        gf_download(self.h, lat, ptr, dev)
        return out

    def functional_theta(self):
        return gf_functional_theta(self.h)

    def or_sweep(self, parity: int = 2, omega: float = 1.7):
        gf_or_sweep(self.h, parity, omega)

    def fix(self, eps: float, maxiter: int, history: int = 0):
        """gf_fix; history > 0 also returns up to that many records (sweep, then F and
        theta of every lattice) of the checks, as an array under "history"."""
        buf = None
        if history > 0:
            import torch
            buf = torch.zeros((history, 1 + 2 * len(self.dims_list)), dtype=torch.float64,
                              device=self.device)
            gf_set_history(self.h, buf.data_ptr(), history)
        try:
            rc, it, F, th = gf_fix(self.h, eps, maxiter)
            out = dict(rc=rc, iters=it, F=F, theta=th, phase_sweeps=gf_fix_phase_sweeps(self.h))
            if buf is not None:
                n = gf_history_count(self.h)
                out["history"] = buf[:n].cpu().numpy()
        finally:
            if buf is not None:
                gf_set_history(self.h, 0, 0)
        return out
