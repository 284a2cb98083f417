"""Thin Python binding of libbras (argument marshalling only).

Every numerical step runs inside ``libbras.so`` (sm_103a CUDA kernels); this module only
converts torch tensors to raw pointers and checks return codes.  If the shared library is
missing the import fails loudly: there is no Python or CPU fallback.

Low-level functions carry the C names (``bras_setup``, ``bras_apply``, ...); ``Context`` is a
small convenience wrapper around one ``bras_ctx``.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbras.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "bras.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2607_12138_b300.build`")
_lib = ctypes.CDLL(LIB_PATH)

H1, HCURL, HDIV = 0, 1, 2
FP64, FP32, BF16, FP64X = 0, 1, 2, 3
PC_NONE, PC_JACOBI, PC_BRAS = 0, 1, 2
SOLVE_FP64, SOLVE_MIXED = 0, 1
# h1b: H1 with the Bernstein basis; h1g: H1 Lagrange at GLL-based nodes (the paper's nodal
# variant); n2curl / bdm: the second-kind H(curl) / H(div) families
SPACES = {"h1": H1, "hcurl": HCURL, "hdiv": HDIV, "h1b": H1, "h1g": H1, "n2curl": HCURL, "bdm": HDIV}
BASIS = {"h1b": 1, "n2curl": 1, "bdm": 1, "h1g": 2}

OK, NOT_CONVERGED = 0, 1
ERR = {-1: "INVALID", -2: "L2G_RANGE", -3: "NO_COPY", -4: "DEGENERATE", -5: "NOT_SPD", -6: "CUDA",
       -7: "OOM", -8: "BREAKDOWN", -9: "PRECISION", -10: "TOO_LARGE", -11: "DEVICE"}


class BrasError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        self.detail = int(_lib.bras_last_error_detail())
        super().__init__(f"{where}: {bras_status_string(code)} (code {code}, detail {self.detail})")


class bras_options(ctypes.Structure):
    _fields_ = [("precisions", ctypes.c_int), ("block_elems", ctypes.c_int), ("max_nrhs", ctypes.c_int),
                ("simt_only", ctypes.c_int), ("basis", ctypes.c_int), ("autotune", ctypes.c_int)]


_vp, _i64, _int, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
_lib.bras_setup.argtypes = [ctypes.POINTER(_vp), _int, _int, _int, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _vp,
                            ctypes.POINTER(bras_options), _vp]
_lib.bras_setup.restype = _int
_lib.bras_n_local.argtypes = [_int, _int, _int, _int]
_lib.bras_n_local.restype = _int
for _name in ("bras_mass_apply", "bras_apply", "bras_apply_noalloc", "bras_jacobi_apply"):
    getattr(_lib, _name).argtypes = [_vp, _int, _vp, _vp, _int, _vp]
    getattr(_lib, _name).restype = _int
_lib.bras_pcg_solve.argtypes = [_vp, _int, _int, _int, _vp, _vp, _int, _dbl, _int, _vp, _vp, _vp]
_lib.bras_pcg_solve.restype = _int
_lib.bras_lambda_max.argtypes = [_vp, _int, _vp, _int, _int, _vp, _vp]
_lib.bras_lambda_max.restype = _int
_lib.bras_fixed_point_solve.argtypes = [_vp, _int, _vp, _vp, _vp, _int, _dbl, _int, _vp, _vp, _vp]
_lib.bras_fixed_point_solve.restype = _int
_lib.bras_chebyshev_solve.argtypes = [_vp, _int, _vp, _vp, _vp, _vp, _int, _dbl, _int, _vp, _vp, _vp]
_lib.bras_chebyshev_solve.restype = _int
_lib.bras_cg_lanczos.argtypes = [_vp, _int, _vp, _int, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), ctypes.POINTER(_int), _vp]
_lib.bras_cg_lanczos.restype = _int
_lib.bras_schur_apply.argtypes = [_vp, _int, _vp, _vp, _vp]
_lib.bras_schur_apply.restype = _int
_lib.bras_grad_rho.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.bras_grad_rho.restype = _int
_lib.bras_update_rho.argtypes = [_vp, _vp, _vp]
_lib.bras_update_rho.restype = _int
_lib.bras_grad_log_rho.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.bras_grad_log_rho.restype = _int
_lib.bras_update_log_rho.argtypes = [_vp, _vp, _vp]
_lib.bras_update_log_rho.restype = _int
_lib.bras_block_tuning.argtypes = [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int), _vp, _vp]
_lib.bras_block_tuning.restype = _int
_lib.bras_info.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_int), ctypes.POINTER(_int)]
_lib.bras_info.restype = _int
_lib.bras_algorithmic_bytes.argtypes = [_vp, _int, _int, _int]
_lib.bras_algorithmic_bytes.restype = _i64
class bras_mesh_desc(ctypes.Structure):
    _fields_ = [("n_vert", _i64), ("coords", _vp), ("n_cell", _i64), ("cells", _vp), ("n_dof", _i64),
                ("l2g", _vp), ("signs", _vp), ("rho", _vp)]


_lib.bras_setup_batched.argtypes = [ctypes.POINTER(_vp), _int, _int, _int, _int, ctypes.POINTER(bras_mesh_desc),
                                    ctypes.POINTER(bras_options), _vp]
_lib.bras_setup_batched.restype = _int
_lib.bras_batch_offsets.argtypes = [_vp, ctypes.POINTER(_int), _vp]
_lib.bras_batch_offsets.restype = _int
_lib.bras_destroy.argtypes = [_vp]
_lib.bras_destroy.restype = None
_lib.bras_status_string.argtypes = [_int]
_lib.bras_status_string.restype = ctypes.c_char_p
_lib.bras_last_error_detail.argtypes = []
_lib.bras_last_error_detail.restype = _i64
_lib.bras_kernel_launches.argtypes = []
_lib.bras_kernel_launches.restype = _i64
_lib.bras_graph_launches.argtypes = []
_lib.bras_graph_launches.restype = _i64
_lib.bras_device_status.argtypes = [_vp, _vp, _int]
_lib.bras_device_status.restype = _int
_lib.bras_wait_selftest.argtypes = [ctypes.POINTER(_int), ctypes.POINTER(_dbl)]
_lib.bras_wait_selftest.restype = _int


def kernel_launches() -> int:
    """CUDA kernels the library has launched since it was loaded (graph-run kernels included)."""
    return int(_lib.bras_kernel_launches())


def graph_launches() -> int:
    """CUDA graph launches the library has made since it was loaded (one per graph-run solve)."""
    return int(_lib.bras_graph_launches())


def bras_wait_selftest() -> tuple[int, float]:
    """One bounded wait on a barrier nothing completes: (status bits recorded, duration ms)."""
    bits, ms = _int(0), _dbl(0.0)
    _check(_lib.bras_wait_selftest(ctypes.byref(bits), ctypes.byref(ms)), "bras_wait_selftest")
    return int(bits.value), float(ms.value)


def bras_device_status(ctx, stream=None, clear: bool = True) -> tuple[int, int]:
    """(return code, status bits) of the context's device status word; BRAS_ERR_DEVICE if set."""
    rc = int(_lib.bras_device_status(ctx, _stream(stream), 1 if clear else 0))
    return rc, int(_lib.bras_last_error_detail()) if rc == -11 else 0


def header_functions() -> list[str]:
    """Names of the functions declared in include/bras.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bras_[a-z0-9_]+)\s*\(", txt)))


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    raise TypeError(type(t))


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise BrasError(rc, where)
    return rc


# ---- low-level names (same as the C ABI) -------------------------------------------------
def bras_status_string(code: int) -> str:
    return _lib.bras_status_string(code).decode()


def bras_n_local(dim: int, space: int, order: int, basis: int = 0) -> int:
    return _lib.bras_n_local(dim, space, order, basis)


def bras_setup(dim, space, order, coords, cells, n_dof, l2g, signs=None, rho=None, options=None, stream=None):
    ctx = _vp()
    opt = options or bras_options(0, 0, 1, 0)
    rc = _lib.bras_setup(ctypes.byref(ctx), dim, space, order, coords.shape[0], _ptr(coords), cells.shape[0],
                         _ptr(cells), n_dof, _ptr(l2g), _ptr(signs), _ptr(rho), ctypes.byref(opt), _stream(stream))
    _check(rc, "bras_setup")
    return ctx


def bras_setup_batched(dim, space, order, meshes, options=None, stream=None):
    """meshes: list of dicts with torch/numpy arrays coords, cells, l2g and optional signs, rho
    and the integer n_dof (the arrays must stay alive during the call)."""
    descs = (bras_mesh_desc * len(meshes))()
    for i, m in enumerate(meshes):
        descs[i] = bras_mesh_desc(m["coords"].shape[0], _ptr(m["coords"]), m["cells"].shape[0], _ptr(m["cells"]),
                                  int(m["n_dof"]), _ptr(m["l2g"]), _ptr(m.get("signs")), _ptr(m.get("rho")))
    ctx = _vp()
    opt = options or bras_options(0, 0, 1, 0)
    rc = _lib.bras_setup_batched(ctypes.byref(ctx), dim, space, order, len(meshes), descs, ctypes.byref(opt),
                                 _stream(stream))
    _check(rc, "bras_setup_batched")
    return ctx


def bras_batch_offsets(ctx):
    n = _int()
    _check(_lib.bras_batch_offsets(ctx, ctypes.byref(n), None), "bras_batch_offsets")
    off = np.zeros(n.value + 1, dtype=np.int64)
    _check(_lib.bras_batch_offsets(ctx, ctypes.byref(n), off.ctypes.data), "bras_batch_offsets")
    return off


def bras_mass_apply(ctx, precision, x, y, nrhs=1, stream=None):
    return _check(_lib.bras_mass_apply(ctx, precision, _ptr(x), _ptr(y), nrhs, _stream(stream)), "bras_mass_apply")


def bras_apply(ctx, precision, x, y, nrhs=1, stream=None):
    return _check(_lib.bras_apply(ctx, precision, _ptr(x), _ptr(y), nrhs, _stream(stream)), "bras_apply")


def bras_apply_noalloc(ctx, precision, x, y, nrhs=1, stream=None):
    """bras_apply without any device allocation (fixed library-owned scratch; see bras.h)."""
    return _check(_lib.bras_apply_noalloc(ctx, precision, _ptr(x), _ptr(y), nrhs, _stream(stream)),
                  "bras_apply_noalloc")


def bras_jacobi_apply(ctx, precision, x, y, nrhs=1, stream=None):
    return _check(_lib.bras_jacobi_apply(ctx, precision, _ptr(x), _ptr(y), nrhs, _stream(stream)), "bras_jacobi_apply")


def bras_pcg_solve(ctx, pc, mode, inner_precision, b, x, nrhs, rtol, maxit, iters, relres, stream=None):
    rc = _lib.bras_pcg_solve(ctx, pc, mode, inner_precision, _ptr(b), _ptr(x), nrhs, rtol, maxit, _ptr(iters),
                             _ptr(relres), _stream(stream))
    return _check(rc, "bras_pcg_solve")


def bras_lambda_max(ctx, pc, v0, nrhs, iters, lam, stream=None):
    return _check(_lib.bras_lambda_max(ctx, pc, _ptr(v0), nrhs, iters, _ptr(lam), _stream(stream)), "bras_lambda_max")


def bras_fixed_point_solve(ctx, pc, omega, b, x, nrhs, rtol, maxit, iters, relres, stream=None):
    rc = _lib.bras_fixed_point_solve(ctx, pc, _ptr(omega), _ptr(b), _ptr(x), nrhs, rtol, maxit, _ptr(iters),
                                     _ptr(relres), _stream(stream))
    return _check(rc, "bras_fixed_point_solve")


def bras_chebyshev_solve(ctx, pc, lmin, lmax, b, x, nrhs, rtol, maxit, iters, relres, stream=None):
    rc = _lib.bras_chebyshev_solve(ctx, pc, _ptr(lmin), _ptr(lmax), _ptr(b), _ptr(x), nrhs, rtol, maxit, _ptr(iters),
                                   _ptr(relres), _stream(stream))
    return _check(rc, "bras_chebyshev_solve")


def bras_cg_lanczos(ctx, pc, b, steps, stream=None):
    """(lambda_min, lambda_max, steps done) of Mt^{-1} M from CG-Lanczos."""
    lo, hi, k = _dbl(), _dbl(), _int()
    _check(_lib.bras_cg_lanczos(ctx, pc, _ptr(b), steps, ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(k),
                                _stream(stream)), "bras_cg_lanczos")
    return lo.value, hi.value, k.value


def bras_schur_apply(ctx, precision, x, y, stream=None):
    return _check(_lib.bras_schur_apply(ctx, precision, _ptr(x), _ptr(y), _stream(stream)), "bras_schur_apply")


def bras_grad_rho(ctx, x, lam, rho_bar, stream=None):
    return _check(_lib.bras_grad_rho(ctx, _ptr(x), _ptr(lam), _ptr(rho_bar), _stream(stream)), "bras_grad_rho")


def bras_update_rho(ctx, rho, stream=None):
    return _check(_lib.bras_update_rho(ctx, _ptr(rho), _stream(stream)), "bras_update_rho")


def bras_grad_log_rho(ctx, x, lam, z_bar, stream=None):
    return _check(_lib.bras_grad_log_rho(ctx, _ptr(x), _ptr(lam), _ptr(z_bar), _stream(stream)), "bras_grad_log_rho")


def bras_update_log_rho(ctx, z, stream=None):
    return _check(_lib.bras_update_log_rho(ctx, _ptr(z), _stream(stream)), "bras_update_log_rho")


def bras_info(ctx):
    n, e, nl, nb = _i64(), _i64(), _int(), _int()
    _check(_lib.bras_info(ctx, ctypes.byref(n), ctypes.byref(e), ctypes.byref(nl), ctypes.byref(nb)), "bras_info")
    return n.value, e.value, nl.value, nb.value


def bras_block_tuning(ctx):
    """(block size in use, [(size, BRAS apply us), ...] timed by the autotuner)."""
    be, cnt = _int(), _int()
    sizes = np.zeros(8, dtype=np.int32)
    us = np.zeros(8, dtype=np.float32)
    _check(_lib.bras_block_tuning(ctx, ctypes.byref(be), ctypes.byref(cnt), sizes.ctypes.data, us.ctypes.data),
           "bras_block_tuning")
    return be.value, [(int(sizes[i]), float(us[i])) for i in range(cnt.value)]


def bras_algorithmic_bytes(ctx, precision, nrhs, bras):
    return int(_lib.bras_algorithmic_bytes(ctx, precision, nrhs, int(bras)))


def bras_destroy(ctx):
    _lib.bras_destroy(ctx)


def bras_last_error_detail() -> int:
    return int(_lib.bras_last_error_detail())


# ---- convenience wrapper -----------------------------------------------------------------
class Context:
    """One BRAS context on the current CUDA device (tensors in, tensors out)."""

    def __init__(self, coords, cells, space: str, order: int, n_dof: int, l2g, signs=None, rho=None,
                 precisions: int = 0, block_elems: int = 0, max_nrhs: int = 1, simt_only: bool = False,
                 autotune: bool = False, stream=None):
        dev = torch.device("cuda")
        self.dim = coords.shape[1]
        self.space = SPACES[space]
        self.order = order
        self.n_dof = int(n_dof)
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(dev) if a is not None else None
        self._coords = t(coords, torch.float64)
        self._cells = t(cells, torch.int32)
        self._l2g = t(l2g, torch.int32)
        self._signs = t(signs, torch.int8)
        self._rho = t(rho, torch.float64)
        self.n_cell = int(self._cells.shape[0])
        opt = bras_options(precisions, block_elems, max_nrhs, int(simt_only), BASIS.get(space, 0), int(autotune))
        self.ctx = bras_setup(self.dim, self.space, order, self._coords, self._cells, self.n_dof, self._l2g,
                              self._signs, self._rho, opt, stream)
        _, _, self.n_loc, self.n_blocks = bras_info(self.ctx)

    @classmethod
    def batched(cls, meshes, space: str, order: int, precisions: int = 0, block_elems: int = 0, autotune: bool = False,
                stream=None):
        """One context over several independent meshes: ``meshes`` is a list of
        (coords, cells, n_dof, l2g, signs) tuples (numpy); vectors are concatenated per mesh."""
        self = cls.__new__(cls)
        keep = []
        descs = []
        for coords, cells, n_dof, l2g, signs in meshes:
            d = {"coords": np.ascontiguousarray(coords, dtype=np.float64),
                 "cells": np.ascontiguousarray(cells, dtype=np.int32),
                 "l2g": np.ascontiguousarray(l2g, dtype=np.int32), "n_dof": int(n_dof),
                 "signs": None if signs is None else np.ascontiguousarray(signs, dtype=np.int8)}
            keep.append(d)
            descs.append(d)
        self.dim = meshes[0][0].shape[1]
        self.space = SPACES[space]
        self.order = order
        opt = bras_options(precisions, block_elems, 1, 0, BASIS.get(space, 0), int(autotune))
        self.ctx = bras_setup_batched(self.dim, self.space, order, descs, opt, stream)
        self.offsets = bras_batch_offsets(self.ctx)
        self.n_dof, self.n_cell, self.n_loc, self.n_blocks = bras_info(self.ctx)
        self.n_mesh = len(meshes)
        return self

    def device_status(self, stream=None, clear: bool = True) -> tuple[int, int]:
        """(return code, status bits) of this context's bounded kernel waits."""
        return bras_device_status(self.ctx, stream, clear)

    @property
    def block_tuning(self):
        """(block size in use, [(size, BRAS apply us), ...] timed by the autotuner)."""
        return bras_block_tuning(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            bras_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _dtype(precision):
        return torch.float64 if precision in (FP64, FP64X) else torch.float32

    def _apply(self, fn, x, precision, out=None, stream=None):
        x = x.contiguous()
        nrhs = 1 if x.dim() == 1 else x.shape[1]
        y = out if out is not None else torch.empty_like(x)
        fn(self.ctx, precision, x, y, nrhs, stream)
        return y

    def mass_apply(self, x, precision=FP64, out=None, stream=None):
        return self._apply(bras_mass_apply, x, precision, out, stream)

    def bras_apply(self, x, precision=FP64, out=None, stream=None):
        return self._apply(bras_apply, x, precision, out, stream)

    def jacobi_apply(self, x, precision=FP64, out=None, stream=None):
        return self._apply(bras_jacobi_apply, x, precision, out, stream)

    def _slot_array(self, v, nrhs):
        slots = max(nrhs, getattr(self, "n_mesh", 1))
        return np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float64), (slots,)))

    def lambda_max(self, v0, pc=PC_BRAS, iters=100, stream=None):
        """Power-iteration lambda_max(Mt^{-1} M) from the start vector(s) v0 (float64 tensor)."""
        nrhs = 1 if v0.dim() == 1 else v0.shape[1]
        lam = np.zeros(max(nrhs, getattr(self, "n_mesh", 1)), dtype=np.float64)
        bras_lambda_max(self.ctx, pc, v0, nrhs, iters, lam, stream)
        return lam

    def schur_apply(self, x, precision=FP64, out=None, stream=None):
        """y = B M_bras^{-1} B^T x for RT_k / DG_{k-1} (x: n_cell * k(k+1)(k+2)/6 values)."""
        y = out if out is not None else torch.empty_like(x)
        bras_schur_apply(self.ctx, precision, x, y, stream)
        return y

    def cg_lanczos(self, b, pc=PC_BRAS, steps=100, stream=None):
        """(lambda_min, lambda_max, steps done) estimates of Mt^{-1} M; kappa_hat = ratio."""
        return bras_cg_lanczos(self.ctx, pc, b, steps, stream)

    def fixed_point_solve(self, b, omega, pc=PC_BRAS, rtol=1e-10, maxit=5000, out=None, stream=None):
        """Damped fixed point; omega scalar or per rhs.  Returns (x, iters, relres, status)."""
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        x = out if out is not None else torch.empty_like(b)
        om = self._slot_array(omega, nrhs)
        iters = np.zeros(om.size, dtype=np.int32)
        relres = np.zeros(om.size, dtype=np.float64)
        st = bras_fixed_point_solve(self.ctx, pc, om, b, x, nrhs, rtol, maxit, iters, relres, stream)
        return x, iters, relres, st

    def chebyshev_solve(self, b, lmin, lmax, pc=PC_BRAS, rtol=1e-10, maxit=5000, out=None, stream=None):
        """Chebyshev semi-iteration on [lmin, lmax].  Returns (x, iters, relres, status)."""
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        x = out if out is not None else torch.empty_like(b)
        lo, hi = self._slot_array(lmin, nrhs), self._slot_array(lmax, nrhs)
        iters = np.zeros(lo.size, dtype=np.int32)
        relres = np.zeros(lo.size, dtype=np.float64)
        st = bras_chebyshev_solve(self.ctx, pc, lo, hi, b, x, nrhs, rtol, maxit, iters, relres, stream)
        return x, iters, relres, st

    def pcg_solve(self, b, pc=PC_BRAS, mode=SOLVE_FP64, inner_precision=FP32, rtol=1e-10, maxit=5000,
                  out=None, stream=None):
        """Returns (x, iters, relres, status); b/x may be CUDA or CPU float64 tensors."""
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        x = out if out is not None else torch.empty_like(b)
        slots = max(nrhs, getattr(self, "n_mesh", 1))
        iters = np.zeros(slots, dtype=np.int32)
        relres = np.zeros(slots, dtype=np.float64)
        st = bras_pcg_solve(self.ctx, pc, mode, inner_precision, b, x, nrhs, rtol, maxit, iters, relres, stream)
        return x, iters, relres, st

    def grad_rho(self, x, lam, stream=None):
        out = torch.empty(self.n_cell, dtype=torch.float64, device=x.device)
        bras_grad_rho(self.ctx, x.contiguous(), lam.contiguous(), out, stream)
        return out

    def update_rho(self, rho, stream=None):
        self._rho = torch.as_tensor(rho, dtype=torch.float64, device="cuda").contiguous()
        bras_update_rho(self.ctx, self._rho, stream)

    def grad_log_rho(self, x, lam, stream=None):
        """z_bar = rho_bar * rho for the log-densities z (rho = exp(z)), computed in the library."""
        out = torch.empty(self.n_cell, dtype=torch.float64, device=x.device)
        bras_grad_log_rho(self.ctx, x.contiguous(), lam.contiguous(), out, stream)
        return out

    def update_log_rho(self, z, stream=None):
        """Element weights rho = exp(z), exponentiated on the device by the library."""
        self._rho = torch.as_tensor(z, dtype=torch.float64, device="cuda").contiguous()
        bras_update_log_rho(self.ctx, self._rho, stream)

    def algorithmic_bytes(self, precision, nrhs=1, bras=True):
        return bras_algorithmic_bytes(self.ctx, precision, nrhs, bras)
