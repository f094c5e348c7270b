"""Thin ctypes binding of libakra.so (the C ABI in include/akra.h).

Argument marshalling only: every step of the operator chain and of the solver runs in the
library's CUDA kernels.  Tensors are torch CUDA tensors (device memory and streams); the
functions keep the C names.  There is no CPU fallback: without the built library on a CUDA
device every call raises.

Layouts (see include/akra.h):
  alm  [R, 2, ntri] complex128 (F64) / complex64 (F32), packed m-major, (E, B)
  maps [R, 2, npix] float64 / float32, RING order, (γ1, γ2)
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

F64, F32, MIXED = 0, 1, 2
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ENUMERIC",
           6: "ETIMEOUT", 7: "ENOWEIGHTS"}


class AkraError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class CgInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer", ctypes.c_int), ("h_applies_f64", ctypes.c_int),
                ("h_applies_f32", ctypes.c_int), ("relres", ctypes.c_double), ("status", ctypes.c_int),
                ("relres_rhs", ctypes.POINTER(ctypes.c_double)), ("iters_rhs", ctypes.POINTER(ctypes.c_int))]


class PlanDesc(ctypes.Structure):
    _fields_ = [("nside", ctypes.c_int), ("lmax", ctypes.c_int), ("nring", ctypes.c_int),
                ("nunit", ctypes.c_int), ("npix", ctypes.c_longlong), ("ntri", ctypes.c_longlong),
                ("has_weights", ctypes.c_int), ("n_active_rings", ctypes.c_int),
                ("n_active_units", ctypes.c_int),
                ("lambda_", ctypes.c_double), ("lambda_eff", ctypes.c_double),
                ("precond", ctypes.c_double), ("omega", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("kernel_launches", ctypes.c_longlong),
                ("legendre_steps_f32", ctypes.c_longlong), ("legendre_steps_f64", ctypes.c_longlong),
                ("legendre_steps_f32_one_ring", ctypes.c_longlong),
                ("legendre_steps_f64_one_ring", ctypes.c_longlong)]


EXPORTS = ["akra_plan_create", "akra_plan_destroy", "akra_last_error", "akra_version",
           "akra_plan_describe", "akra_plan_set_weights", "akra_synth_spin2",
           "akra_adjoint_synth_spin2", "akra_apply_A", "akra_apply_At", "akra_apply_H",
           "akra_cg_solve", "akra_cg_solve_b", "akra_set_timeout", "akra_autotune",
           "akra_time_H_stages", "akra_synth_spin2_static", "akra_cg_solve_adjoint",
           "akra_weight_grad", "akra_batch_create", "akra_batch_destroy", "akra_batch_autotune",
           "akra_batch_apply_H", "akra_batch_cg_solve", "akra_batch_describe",
           "akra_plan_get_shape", "akra_plan_set_shape", "akra_set_mixed_policy", "akra_fma_rate",
           "akra_cg_solve_fields", "akra_shuffle_shear", "akra_cl_spectra",
           "akra_plan_set_preconditioner", "akra_flat_plan_create", "akra_plan_fill_workspaces",
           "akra_debug_violations", "akra_plan_set_tc_synthesis", "akra_plan_get_tc_synthesis",
           "akra_batch_set_tc_synthesis", "akra_batch_get_tc_synthesis", "akra_legendre_lane_steps",
           "akra_plan_set_adjoint_shape", "akra_plan_get_adjoint_shape"]

_lib_handle = None


def library_path() -> str:
    """libakra.so in the package directory, or the file named by AKRA_LIBRARY (e.g. the
    bounds-checked debug build libakra_debug.so)."""
    return os.environ.get("AKRA_LIBRARY") or _build.OUT


def load(build_if_missing: bool = False):
    """Load libakra.so (raises if it is missing; never falls back to anything else)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing or path != _build.OUT:
            raise RuntimeError("%s is not built (run paper_2606_06175_gb300/build.py)" % path)
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "akra_plan_create": ([i, i, ctypes.POINTER(vp)], i),
        "akra_flat_plan_create": ([i, ctypes.POINTER(vp)], i),
        "akra_plan_destroy": ([vp], None),
        "akra_last_error": ([], ctypes.c_char_p),
        "akra_version": ([], ctypes.c_char_p),
        "akra_plan_describe": ([vp, ctypes.POINTER(PlanDesc)], i),
        "akra_plan_set_weights": ([vp, vp, d, vp], i),
        "akra_synth_spin2": ([vp, i, vp, vp, i, vp], i),
        "akra_adjoint_synth_spin2": ([vp, i, vp, vp, i, vp], i),
        "akra_apply_A": ([vp, i, vp, vp, i, i, vp], i),
        "akra_apply_At": ([vp, i, vp, vp, i, i, vp], i),
        "akra_apply_H": ([vp, i, vp, vp, i, vp], i),
        "akra_cg_solve": ([vp, i, vp, vp, i, d, i, ctypes.POINTER(CgInfo), vp], i),
        "akra_cg_solve_b": ([vp, i, vp, vp, i, d, i, ctypes.POINTER(CgInfo), vp], i),
        "akra_cg_solve_fields": ([vp, i, i, vp, vp, i, d, i, ctypes.POINTER(CgInfo), vp], i),
        "akra_set_timeout": ([d], i),
        "akra_set_mixed_policy": ([d, d], i),
        "akra_plan_set_preconditioner": ([vp, i], i),
        "akra_plan_fill_workspaces": ([vp, i, vp], i),
        "akra_debug_violations": ([ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(i),
                                   ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)], i),
        "akra_shuffle_shear": ([vp, i, vp, vp, vp, i, vp], i),
        "akra_cl_spectra": ([vp, i, vp, vp, i, i, ctypes.POINTER(d), vp, vp], i),
        "akra_fma_rate": ([i, ctypes.POINTER(d)], i),
        "akra_autotune": ([vp, i, i, vp], i),
        "akra_plan_get_shape": ([vp, i, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)], i),
        "akra_plan_set_shape": ([vp, i, i, i, i, i], i),
        "akra_plan_set_tc_synthesis": ([vp, i, i], i),
        "akra_plan_get_tc_synthesis": ([vp, i, ctypes.POINTER(i)], i),
        "akra_batch_set_tc_synthesis": ([vp, i], i),
        "akra_batch_get_tc_synthesis": ([vp, ctypes.POINTER(i)], i),
        "akra_legendre_lane_steps": ([vp, i, i, i, i, ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_longlong)], i),
        "akra_plan_set_adjoint_shape": ([vp, i, i, i, i], i),
        "akra_plan_get_adjoint_shape": ([vp, i, i, ctypes.POINTER(i), ctypes.POINTER(i)], i),
        "akra_time_H_stages": ([vp, i, i, i, vp, ctypes.POINTER(ctypes.c_double)], i),
        "akra_synth_spin2_static": ([vp, i, vp, vp, i, vp], i),
        "akra_cg_solve_adjoint": ([vp, i, vp, vp, i, d, i, ctypes.POINTER(CgInfo), vp], i),
        "akra_weight_grad": ([vp, i, vp, vp, vp, vp, i, vp], i),
        "akra_batch_create": ([i, ctypes.POINTER(vp), ctypes.POINTER(i), ctypes.POINTER(vp)], i),
        "akra_batch_destroy": ([vp], None),
        "akra_batch_autotune": ([vp, vp], i),
        "akra_batch_apply_H": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp], i),
        "akra_batch_cg_solve": ([vp, i, ctypes.POINTER(vp), ctypes.POINTER(vp), d, i,
                                 ctypes.POINTER(CgInfo), vp], i),
        "akra_batch_describe": ([vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong)], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib_handle = lib
    return lib


def _check(status: int):
    if status != 0:
        raise AkraError(status, load().akra_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """Owning handle of an akra_plan (nside, lmax)."""

    def __init__(self, handle, nside, lmax):
        self.handle = handle
        self.nside = nside
        self.lmax = lmax
        self.npix = 12 * nside * nside
        self.ntri = (lmax + 1) * (lmax + 2) // 2

    def alm_shape(self, R: int):
        """Shape of R harmonic vectors: [R, 2, ntri] (E, B) packed m-major."""
        return (R, 2, self.ntri)

    def close(self):
        if self.handle:
            load().akra_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _cdtype(prec):
    return torch.complex128 if prec == F64 else torch.complex64


def _rdtype(prec):
    return torch.float64 if prec == F64 else torch.float32


def _need(t: torch.Tensor, shape, dtype, name):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and tuple(t.shape) == tuple(shape)):
        raise ValueError("%s must be a contiguous CUDA %s tensor of shape %s (got %s %s %s)"
                         % (name, dtype, tuple(shape), t.device, t.dtype, tuple(t.shape)))


def akra_version() -> str:
    return load().akra_version().decode()


def akra_plan_create(nside: int, lmax: int) -> Plan:
    h = ctypes.c_void_p()
    _check(load().akra_plan_create(nside, lmax, ctypes.byref(h)))
    return Plan(h, nside, lmax)


class FlatPlan(Plan):
    """Owning handle of a flat-sky plan on an n x n periodic grid: harmonic vectors are
    [R, n, n] complex (the unitary 2D FFT of κ_E + i κ_B), maps [R, 2, n*n]."""

    def __init__(self, handle, n):
        super().__init__(handle, n, -1)
        self.n = n
        self.npix = n * n
        self.ntri = n * n // 2

    def alm_shape(self, R: int):
        return (R, self.n, self.n)


def akra_flat_plan_create(n: int) -> FlatPlan:
    h = ctypes.c_void_p()
    _check(load().akra_flat_plan_create(n, ctypes.byref(h)))
    return FlatPlan(h, n)


def akra_plan_destroy(plan: Plan):
    plan.close()


def akra_plan_describe(plan: Plan) -> dict:
    d = PlanDesc()
    _check(load().akra_plan_describe(plan.handle, ctypes.byref(d)))
    return {f: getattr(d, f) for f, _ in PlanDesc._fields_}


def akra_debug_violations() -> dict:
    """Out-of-bounds accesses recorded by the debug build since the last call (count -1: the
    release build, which has no checks); clears the record."""
    c, si = ctypes.c_longlong(), ctypes.c_int()
    ix, bd = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load().akra_debug_violations(ctypes.byref(c), ctypes.byref(si), ctypes.byref(ix), ctypes.byref(bd)))
    return {"count": c.value, "site": si.value, "index": ix.value, "bound": bd.value}


def akra_plan_fill_workspaces(plan: Plan, byte: int = 0xFF, stream=None):
    """Fill every workspace the plan holds with `byte` (0xFF: NaN in FP32 and FP64), so that a
    later read of an entry no kernel wrote shows up as a non-finite result (testing aid)."""
    _check(load().akra_plan_fill_workspaces(plan.handle, int(byte), _stream(stream)))


def akra_plan_set_weights(plan: Plan, ninv: torch.Tensor, lam: float = 1e-3, stream=None):
    _need(ninv, (plan.npix,), torch.float64, "ninv")
    _check(load().akra_plan_set_weights(plan.handle, _ptr(ninv), float(lam), _stream(stream)))


def akra_synth_spin2(plan: Plan, prec: int, alm: torch.Tensor, out: torch.Tensor = None, stream=None):
    R = alm.shape[0]
    _need(alm, plan.alm_shape(R), _cdtype(prec), "alm")
    if out is None:
        out = torch.empty((R, 2, plan.npix), dtype=_rdtype(prec), device=alm.device)
    _need(out, (R, 2, plan.npix), _rdtype(prec), "out")
    _check(load().akra_synth_spin2(plan.handle, prec, _ptr(alm), _ptr(out), R, _stream(stream)))
    return out


def akra_synth_spin2_static(plan: Plan, prec: int, alm: torch.Tensor, out: torch.Tensor, stream=None):
    """akra_synth_spin2 that allocates no device memory (the caller passes `out`; the
    library's fixed 32 MiB scratch holds the phase array).  For callers that cannot allocate
    at the point of the call, e.g. inside a stream capture or under an allocation budget."""
    R = alm.shape[0]
    _need(alm, plan.alm_shape(R), _cdtype(prec), "alm")
    _need(out, (R, 2, plan.npix), _rdtype(prec), "out")
    _check(load().akra_synth_spin2_static(plan.handle, prec, _ptr(alm), _ptr(out), R, _stream(stream)))
    return out


def akra_adjoint_synth_spin2(plan: Plan, prec: int, maps: torch.Tensor, out: torch.Tensor = None,
                             stream=None):
    R = maps.shape[0]
    _need(maps, (R, 2, plan.npix), _rdtype(prec), "maps")
    if out is None:
        out = torch.empty(plan.alm_shape(R), dtype=_cdtype(prec), device=maps.device)
    _need(out, plan.alm_shape(R), _cdtype(prec), "out")
    _check(load().akra_adjoint_synth_spin2(plan.handle, prec, _ptr(maps), _ptr(out), R, _stream(stream)))
    return out


def akra_apply_A(plan: Plan, prec: int, x: torch.Tensor, weighted: bool = False, out=None, stream=None):
    R = x.shape[0]
    _need(x, plan.alm_shape(R), _cdtype(prec), "x")
    if out is None:
        out = torch.empty((R, 2, plan.npix), dtype=_rdtype(prec), device=x.device)
    _need(out, (R, 2, plan.npix), _rdtype(prec), "out")
    _check(load().akra_apply_A(plan.handle, prec, _ptr(x), _ptr(out), int(weighted), R, _stream(stream)))
    return out


def akra_apply_At(plan: Plan, prec: int, maps: torch.Tensor, weighted: bool = False, out=None,
                  stream=None):
    R = maps.shape[0]
    _need(maps, (R, 2, plan.npix), _rdtype(prec), "maps")
    if out is None:
        out = torch.empty(plan.alm_shape(R), dtype=_cdtype(prec), device=maps.device)
    _need(out, plan.alm_shape(R), _cdtype(prec), "out")
    _check(load().akra_apply_At(plan.handle, prec, _ptr(maps), _ptr(out), int(weighted), R,
                                _stream(stream)))
    return out


def akra_apply_H(plan: Plan, prec: int, x: torch.Tensor, out: torch.Tensor = None, stream=None):
    R = x.shape[0]
    _need(x, plan.alm_shape(R), _cdtype(prec), "x")
    if out is None:
        out = torch.empty_like(x)
    _need(out, plan.alm_shape(R), _cdtype(prec), "out")
    _check(load().akra_apply_H(plan.handle, prec, _ptr(x), _ptr(out), R, _stream(stream)))
    return out


def _solve(fn, plan, prec, src, out, R, tol, maxiter, stream, raise_on_noconv):
    if out is None:
        out = torch.empty(plan.alm_shape(R), dtype=_cdtype(F64 if prec == MIXED else prec), device=src.device)
    rel = (ctypes.c_double * R)()
    its = (ctypes.c_int * R)()
    info = CgInfo()
    info.relres_rhs = rel
    info.iters_rhs = its
    st = fn(plan.handle, prec, _ptr(src), _ptr(out), R, float(tol), int(maxiter), ctypes.byref(info),
            _stream(stream))
    if st != 0 and (raise_on_noconv or st not in (4, 5)):
        _check(st)
    res = {"iters": info.iters, "outer": info.outer, "h_applies_f64": info.h_applies_f64,
           "h_applies_f32": info.h_applies_f32, "relres": info.relres, "status": st,
           "relres_rhs": list(rel), "iters_rhs": list(its)}
    return out, res


def akra_cg_solve(plan: Plan, prec: int, shear: torch.Tensor, out=None, tol: float = 1e-6,
                  maxiter: int = 1000, stream=None, raise_on_noconv: bool = False):
    R = shear.shape[0]
    _need(shear, (R, 2, plan.npix), torch.float32 if prec == F32 else torch.float64, "shear")
    return _solve(load().akra_cg_solve, plan, prec, shear, out, R, tol, maxiter, stream, raise_on_noconv)


PRECOND_SCALAR, PRECOND_PER_L = 0, 1


def akra_plan_set_preconditioner(plan: Plan, kind: int):
    """PRECOND_SCALAR (Eq. 15, default) or PRECOND_PER_L (per-l diagonal)."""
    _check(load().akra_plan_set_preconditioner(plan.handle, kind))


SOLVE_E, SOLVE_B_GIVEN_E = 1, 2


def akra_cg_solve_fields(plan: Plan, prec: int, fields: int, shear: torch.Tensor, out=None,
                         tol: float = 1e-6, maxiter: int = 1000, stream=None,
                         raise_on_noconv: bool = False):
    """E-only solve (fields=SOLVE_E) or the conditional B-mode solve given κ̂_E in the E field
    of `out` (fields=SOLVE_B_GIVEN_E); see akra_cg_solve_fields in akra.h."""
    R = shear.shape[0]
    _need(shear, (R, 2, plan.npix), torch.float32 if prec == F32 else torch.float64, "shear")
    if fields == SOLVE_B_GIVEN_E:
        if out is None:
            raise ValueError("SOLVE_B_GIVEN_E reads κ_E from `out`")
        _need(out, plan.alm_shape(R), _cdtype(F64 if prec == MIXED else prec), "out")

    def fn(h, pr, src, dst, r, tl, mi, inf, st):
        return load().akra_cg_solve_fields(h, pr, fields, src, dst, r, tl, mi, inf, st)

    return _solve(fn, plan, prec, shear, out, R, tol, maxiter, stream, raise_on_noconv)


def akra_cg_solve_b(plan: Plan, prec: int, b: torch.Tensor, out=None, tol: float = 1e-6,
                    maxiter: int = 1000, stream=None, raise_on_noconv: bool = False):
    R = b.shape[0]
    _need(b, plan.alm_shape(R), _cdtype(F64 if prec == MIXED else prec), "b")
    return _solve(load().akra_cg_solve_b, plan, prec, b, out, R, tol, maxiter, stream, raise_on_noconv)


def akra_cg_solve_adjoint(plan: Plan, prec: int, g: torch.Tensor, out=None, tol: float = 1e-6,
                          maxiter: int = 1000, stream=None, raise_on_noconv: bool = False):
    R = g.shape[0]
    _need(g, plan.alm_shape(R), _cdtype(F64 if prec == MIXED else prec), "g")
    return _solve(load().akra_cg_solve_adjoint, plan, prec, g, out, R, tol, maxiter, stream,
                  raise_on_noconv)


def akra_weight_grad(plan: Plan, prec: int, Au: torch.Tensor, y: torch.Tensor, Ax: torch.Tensor,
                     out: torch.Tensor = None, stream=None):
    R = Au.shape[0]
    dt = _rdtype(prec)
    for t, nm in ((Au, "Au"), (y, "y"), (Ax, "Ax")):
        _need(t, (R, 2, plan.npix), dt, nm)
    if out is None:
        out = torch.empty((plan.npix,), dtype=dt, device=Au.device)
    _need(out, (plan.npix,), dt, "out")
    _check(load().akra_weight_grad(plan.handle, prec, _ptr(Au), _ptr(y), _ptr(Ax), _ptr(out), R,
                                   _stream(stream)))
    return out


def akra_set_timeout(seconds: float):
    _check(load().akra_set_timeout(float(seconds)))


def akra_set_mixed_policy(inner_floor: float = 0.0, inner_factor: float = 0.5):
    """FP32 inner tolerance of mixed-precision solves: max(floor, min(0.1, factor·tol/relres));
    floor 0 = automatic (0.1 · 2^-24 · lmax within [5e-6, 1e-3])."""
    _check(load().akra_set_mixed_policy(float(inner_floor), float(inner_factor)))


def akra_autotune(plan: Plan, prec: int, R: int = 1, stream=None):
    _check(load().akra_autotune(plan.handle, prec, R, _stream(stream)))


def akra_plan_get_shape(plan: Plan, prec: int, R: int = 1) -> dict:
    """Legendre tile shape used for (prec, R): synthesis / adjoint ring pairs per thread, RHS
    per block."""
    P, PA, RG = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().akra_plan_get_shape(plan.handle, prec, R, ctypes.byref(P), ctypes.byref(PA),
                                      ctypes.byref(RG)))
    return {"P": P.value, "PA": PA.value, "RG": RG.value}


def akra_plan_set_adjoint_shape(plan: Plan, prec: int, R: int, PA: int, RGA: int):
    """The adjoint's ring pairs per thread and RHS per block for (prec, R)."""
    _check(load().akra_plan_set_adjoint_shape(plan.handle, prec, R, PA, RGA))


def akra_plan_get_adjoint_shape(plan: Plan, prec: int, R: int = 1) -> dict:
    pa, rga = ctypes.c_int(), ctypes.c_int()
    _check(load().akra_plan_get_adjoint_shape(plan.handle, prec, R, ctypes.byref(pa), ctypes.byref(rga)))
    return {"PA": pa.value, "RGA": rga.value}


def akra_plan_set_tc_synthesis(plan: Plan, R: int, group: int):
    """FP32 synthesis for R RHS on the tensor core with RHS groups of `group` (4, 8, 16, 32), or on
    the CUDA cores (group 0)."""
    _check(load().akra_plan_set_tc_synthesis(plan.handle, R, group))


def akra_plan_get_tc_synthesis(plan: Plan, R: int = 1) -> int:
    g = ctypes.c_int()
    _check(load().akra_plan_get_tc_synthesis(plan.handle, R, ctypes.byref(g)))
    return g.value


def akra_plan_set_shape(plan: Plan, prec: int, R: int, P: int, PA: int, RG: int):
    """Force the Legendre tile shape for (prec, R)."""
    _check(load().akra_plan_set_shape(plan.handle, prec, R, P, PA, RG))


def akra_shuffle_shear(plan: Plan, prec: int, shear: torch.Tensor, perm: torch.Tensor,
                       out: torch.Tensor = None, stream=None) -> torch.Tensor:
    """Gather shear [2, npix] through perm [R, npix] (int32) into [R, 2, npix]."""
    R = perm.shape[0]
    _need(shear, (2, plan.npix), _rdtype(prec), "shear")
    _need(perm, (R, plan.npix), torch.int32, "perm")
    if out is None:
        out = torch.empty((R, 2, plan.npix), dtype=_rdtype(prec), device=shear.device)
    _need(out, (R, 2, plan.npix), _rdtype(prec), "out")
    _check(load().akra_shuffle_shear(plan.handle, prec, _ptr(shear), _ptr(perm), _ptr(out), R,
                                     _stream(stream)))
    return out


def akra_cl_spectra(plan: Plan, prec: int, a: torch.Tensor, b: torch.Tensor = None, edges=None,
                    stream=None) -> torch.Tensor:
    """E/B auto (b = None) or cross spectra [R, 4, lmax+1] (EE, EB, BE, BB), or band powers
    [R, 4, nbins] for the given bin edges."""
    R = a.shape[0]
    _need(a, plan.alm_shape(R), _cdtype(prec), "a")
    if b is None:
        b = a
    _need(b, plan.alm_shape(R), _cdtype(prec), "b")
    nb = 0 if edges is None else len(edges) - 1
    e = (ctypes.c_double * (nb + 1))(*([] if edges is None else [float(v) for v in edges]))
    out = torch.empty((R, 4, nb if nb else plan.lmax + 1), dtype=torch.float64, device=a.device)
    _check(load().akra_cl_spectra(plan.handle, prec, _ptr(a), _ptr(b), R, nb,
                                  e if nb else None, _ptr(out), _stream(stream)))
    return out


def akra_legendre_lane_steps(plan: Plan, prec: int, adjoint: bool, P: int, NT: int = 128) -> dict:
    """Executed lane-steps and counted steps of one Legendre launch with P ring pairs per thread."""
    ls, st = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load().akra_legendre_lane_steps(plan.handle, prec, 1 if adjoint else 0, P, NT,
                                           ctypes.byref(ls), ctypes.byref(st)))
    return {"lane_steps": ls.value, "steps": st.value,
            "efficiency": st.value / ls.value if ls.value else 0.0}


def akra_fma_rate(prec: int) -> float:
    """Measured FMA rate of the current device, TFLOP/s (FP32 or FP64)."""
    v = ctypes.c_double()
    _check(load().akra_fma_rate(prec, ctypes.byref(v)))
    return v.value


def akra_time_H_stages(plan: Plan, prec: int, R: int = 1, reps: int = 3, stream=None) -> dict:
    """Per-stage milliseconds of one H application (CUDA events on `stream`)."""
    ms = (ctypes.c_double * 5)()
    _check(load().akra_time_H_stages(plan.handle, prec, R, reps, _stream(stream), ms))
    return {"legendre_synth": ms[0], "ring_fft": ms[1], "legendre_adjoint": ms[2],
            "epilogue": ms[3], "total": ms[4]}


class Batch:
    """Owning handle of an akra_batch over several plans (kept alive with it)."""

    def __init__(self, handle, plans, R):
        self.handle, self.plans, self.R = handle, list(plans), list(R)

    def close(self):
        if self.handle:
            load().akra_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def akra_batch_create(plans, R) -> Batch:
    n = len(plans)
    arr = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    rr = (ctypes.c_int * n)(*R)
    h = ctypes.c_void_p()
    _check(load().akra_batch_create(n, arr, rr, ctypes.byref(h)))
    return Batch(h, plans, R)


def akra_batch_destroy(batch: Batch):
    batch.close()


def akra_batch_autotune(batch: Batch, stream=None):
    _check(load().akra_batch_autotune(batch.handle, _stream(stream)))


def akra_batch_describe(batch: Batch) -> dict:
    P, RG, nl = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    _check(load().akra_batch_describe(batch.handle, ctypes.byref(P), ctypes.byref(RG), ctypes.byref(nl)))
    return {"P": P.value, "RG": RG.value, "launches": nl.value}


def akra_batch_set_tc_synthesis(batch: Batch, group: int):
    """The batch's FP32 synthesis on the tensor core with RHS groups of `group` (4, 8, 16, 32), or
    on the CUDA cores (group 0)."""
    _check(load().akra_batch_set_tc_synthesis(batch.handle, group))


def akra_batch_get_tc_synthesis(batch: Batch) -> int:
    g = ctypes.c_int()
    _check(load().akra_batch_get_tc_synthesis(batch.handle, ctypes.byref(g)))
    return g.value


def akra_batch_apply_H(batch: Batch, xs, out=None, stream=None):
    n = len(batch.plans)
    if out is None:
        out = [torch.empty_like(x) for x in xs]
    for p, R, x, y in zip(batch.plans, batch.R, xs, out):
        _need(x, (R, 2, p.ntri), torch.complex64, "x")
        _need(y, (R, 2, p.ntri), torch.complex64, "out")
    xa = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    ya = (ctypes.c_void_p * n)(*[y.data_ptr() for y in out])
    _check(load().akra_batch_apply_H(batch.handle, xa, ya, _stream(stream)))
    return out


def akra_batch_cg_solve(batch: Batch, prec: int, shears, out=None, tol: float = 1e-6,
                        maxiter: int = 2000, stream=None, raise_on_noconv: bool = False):
    n = len(batch.plans)
    rdt = torch.float32 if prec == F32 else torch.float64
    cdt = torch.complex64 if prec == F32 else torch.complex128
    if out is None:
        out = [torch.empty((R, 2, p.ntri), dtype=cdt, device=s.device)
               for p, R, s in zip(batch.plans, batch.R, shears)]
    for p, R, y, x in zip(batch.plans, batch.R, shears, out):
        _need(y, (R, 2, p.npix), rdt, "shear")
        _need(x, (R, 2, p.ntri), cdt, "out")
    infos = (CgInfo * n)()
    keep = []
    for k in range(n):
        rel = (ctypes.c_double * batch.R[k])()
        its = (ctypes.c_int * batch.R[k])()
        keep.append((rel, its))
        infos[k].relres_rhs = rel
        infos[k].iters_rhs = its
    ya = (ctypes.c_void_p * n)(*[y.data_ptr() for y in shears])
    xa = (ctypes.c_void_p * n)(*[x.data_ptr() for x in out])
    st = load().akra_batch_cg_solve(batch.handle, prec, ya, xa, float(tol), int(maxiter), infos, _stream(stream))
    if st != 0 and (raise_on_noconv or st not in (4, 5)):
        _check(st)
    res = [{"iters": infos[k].iters, "outer": infos[k].outer, "h_applies_f64": infos[k].h_applies_f64,
            "h_applies_f32": infos[k].h_applies_f32, "relres": infos[k].relres, "status": infos[k].status,
            "relres_rhs": list(keep[k][0]), "iters_rhs": list(keep[k][1])} for k in range(n)]
    return out, res
