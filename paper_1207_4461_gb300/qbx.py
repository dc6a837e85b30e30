"""Thin ctypes binding of the C ABI in include/qbx.h (same names, argument
marshalling only).  Every step of the computation runs in the CUDA library
libqbx_gb300.so; there is no CPU fallback: if the library cannot be built or
loaded, every call raises.

Device arrays are torch tensors (float64 / complex128, contiguous, on the
plan's device); complex128 storage is interleaved (re, im) FP64, the layout of
qbx_c64.  Calls are asynchronous on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np
import torch

from . import build as _build

OP_S, OP_D, OP_GRAD_S, OP_R, OP_GRAD_D = 0, 1, 2, 3, 4
SIDE_INT, SIDE_EXT, SIDE_TWO = 0, 1, 2
LIMIT_ONE_SIDED, LIMIT_PV = 0, 1
VALUE, GRAD = 0, 1
MAX_P = 40

_ERR = {0: "QBX_OK", 1: "QBX_EINVAL", 2: "QBX_ECUDA", 3: "QBX_EINADMISSIBLE", 4: "QBX_ENONFINITE",
        5: "QBX_ENOCONV", 6: "QBX_ETIMEOUT", 7: "QBX_ENOMEM"}


class QBXError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERR.get(code, code)}: {msg}")
        self.code = code


class c64(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


_P = ctypes.c_void_p


class GeomStruct(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("q_tgt", ctypes.c_int), ("q_src", ctypes.c_int),
                ("n_tgt", ctypes.c_int), ("n_src", ctypes.c_int)] + [
        (n, _P) for n in ("src_x", "src_y", "src_nx", "src_ny", "src_w",
                          "tgt_x", "tgt_y", "tgt_nx", "tgt_ny", "tgt_w",
                          "panel_h", "ctr_x", "ctr_y", "ctr_r", "ctr_ratio")]


_lock = threading.Lock()
_lib = None


def lib():
    """Load (building first if needed) the CUDA library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            I, D, Z = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
            G = ctypes.POINTER(GeomStruct)
            PP = ctypes.POINTER(ctypes.c_void_p)
            L.qbx_last_error.restype = ctypes.c_char_p
            L.qbx_version.restype = I
            L.qbx_gauss_legendre.argtypes = [I, _P, _P]
            L.qbx_plan_create.argtypes = [PP, I, I, I, Z]
            L.qbx_plan_destroy.argtypes = [_P]
            L.qbx_workspace_bytes.argtypes = [I, I, I, I]
            L.qbx_workspace_bytes.restype = Z
            L.qbx_sync_status.argtypes = [_P, _P]
            L.qbx_geometry.argtypes = [_P, G, _P, _P, _P, _P, _P, D, _P]
            L.qbx_upsample.argtypes = [_P, G, _P, I, _P, _P]
            L.qbx_form_locals.argtypes = [_P, G, I, I, c64, I, _P, I, _P, _P]
            L.qbx_eval_locals.argtypes = [_P, G, I, c64, I, _P, I, I, I, _P, _P, _P, _P, _P]
            L.qbx_apply.argtypes = [_P, G, I, I, I, c64, I, _P, I, I, _P, _P, _P, _P]
            L.qbx_far.argtypes = [_P, G, I, c64, _P, I, I, _P, _P, _P]
            L.qbx_assign_centres.argtypes = [_P, G, I, I, _P, _P, _P]
            L.qbx_apply_ops.argtypes = [_P, G, I, I, I, c64, I, ctypes.POINTER(_P), I, ctypes.POINTER(_P), _P]
            L.qbx_apply_ops.restype = I
            L.qbx_apply_cfie.argtypes = [_P, G, c64, c64, I, _P, I, _P, _P]
            L.qbx_apply_cfie.restype = I
            L.qbx_batch_create.argtypes = [PP, _P, I, G, ctypes.POINTER(c64), I, I, I, I, I,
                                           ctypes.POINTER(_P), ctypes.POINTER(_P)]
            L.qbx_batch_apply.argtypes = [_P, _P]
            L.qbx_batch_status.argtypes = [_P, _P]
            L.qbx_batch_destroy.argtypes = [_P]
            for name in ("qbx_batch_create", "qbx_batch_apply", "qbx_batch_status", "qbx_batch_destroy"):
                getattr(L, name).restype = I
            L.qbx_solve_exterior_dirichlet.argtypes = [_P, G, c64, c64, I, _P, I, D, I, I, _P,
                                                       ctypes.POINTER(I), ctypes.POINTER(D), _P]
            L.qbx_solve_exterior_dirichlet.restype = I
            L.qbx_apply_adjoint.argtypes = [_P, G, I, I, I, c64, I, _P, I, _P, _P]
            L.qbx_apply_adjoint.restype = I
            L.qbx_apply_shape_adjoint.argtypes = [_P, G, I, c64, I, _P, _P, I, _P, _P, _P, _P, _P, _P, _P]
            L.qbx_apply_shape_adjoint.restype = I
            L.qbx_apply_shape_adjoint_d.argtypes = [_P, G, I, c64, I, _P, _P, I, _P, _P, _P, _P, _P, _P, _P]
            L.qbx_apply_shape_adjoint_d.restype = I
            L.qbx_shape_adjoint_workspace_bytes.argtypes = [I, I, I, I, I]
            L.qbx_batch_tune.argtypes = [_P, _P, ctypes.POINTER(I), ctypes.POINTER(I)]
            L.qbx_batch_tune.restype = I
            L.qbx_batch_info.argtypes = [_P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                         ctypes.POINTER(I)]
            L.qbx_batch_info.restype = I
            L.qbx_batch_set_eta.argtypes = [_P, D]
            L.qbx_batch_set_eta.restype = I
            L.qbx_assemble_cfie.argtypes = [_P, G, c64, c64, I, _P, _P]
            L.qbx_assemble_cfie.restype = I
            L.qbx_solve_exterior_dirichlet_assembled.argtypes = [_P, G, _P, _P, I, D, I, I, _P,
                                                                 ctypes.POINTER(I), ctypes.POINTER(D), _P]
            L.qbx_solve_exterior_dirichlet_assembled.restype = I
            L.qbx_apply_local.argtypes = [_P, G, I, I, I, c64, I, D, ctypes.POINTER(_P), I, ctypes.POINTER(_P), _P]
            L.qbx_apply_local.restype = I
            L.qbx_geometry_rule.argtypes = [_P, G, _P, _P, _P, _P, _P, I, D, _P]
            L.qbx_geometry_rule.restype = I
            L.qbx_plan_set_min_waves.argtypes = [_P, I]
            L.qbx_plan_set_min_waves.restype = I
            L.qbx_plan_set_timing.argtypes = [_P, I]
            L.qbx_plan_set_timing.restype = I
            L.qbx_plan_kernel_ms.argtypes = [_P, ctypes.POINTER(ctypes.c_float)]
            L.qbx_plan_kernel_ms.restype = I
            L.qbx_shape_adjoint_workspace_bytes.restype = ctypes.c_size_t
            L.qbx_apply_static.argtypes = [G, I, I, I, c64, I, _P, I, _P, _P]
            L.qbx_apply_static.restype = I
            L.qbx_matmul_cm.argtypes = [I, I, _P, _P, _P, _P, ctypes.c_size_t, _P]
            L.qbx_matmul_cm.restype = I
            L.qbx_matmul_cm_work_bytes.argtypes = [I, I]
            L.qbx_matmul_cm_work_bytes.restype = ctypes.c_size_t
            L.qbx_apply_static_status.argtypes = [_P]
            L.qbx_apply_static_status.restype = I
            L.qbx_vec_dots.argtypes = [I, I, I, _P, _P, _P, _P, _P]
            L.qbx_vec_dots.restype = I
            L.qbx_vec_dots_work_bytes.argtypes = [I, I]
            L.qbx_vec_dots_work_bytes.restype = Z
            L.qbx_vec_orth_update.argtypes = [I, I, I, _P, _P, _P, _P]
            L.qbx_vec_orth_update.restype = I
            L.qbx_vec_combine.argtypes = [I, I, I, _P, _P, _P, _P]
            L.qbx_vec_combine.restype = I
            L.qbx_debug_hankel01.argtypes = [_P, I, _P, _P, _P]
            L.qbx_debug_besselj.argtypes = [_P, I, I, _P, _P]
            L.qbx_debug_hankel01_ray.argtypes = [_P, c64, _P, I, _P, _P, _P]
            L.qbx_debug_hankel01_ray.restype = I
            for name in ("qbx_gauss_legendre", "qbx_plan_create", "qbx_plan_destroy", "qbx_sync_status",
                         "qbx_geometry", "qbx_upsample", "qbx_form_locals", "qbx_eval_locals", "qbx_apply",
                         "qbx_far", "qbx_assign_centres", "qbx_debug_hankel01", "qbx_debug_besselj"):
                getattr(L, name).restype = I
            _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


def _check(rc):
    if rc != 0:
        raise QBXError(rc, lib().qbx_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _k(k):
    k = complex(k)
    return c64(k.real, k.imag)


# ----------------------------------------------------------------------------
# Host helpers
# ----------------------------------------------------------------------------
def qbx_gauss_legendre(q: int):
    x = np.zeros(q)
    w = np.zeros(q)
    _check(lib().qbx_gauss_legendre(q, x.ctypes.data_as(_P), w.ctypes.data_as(_P)))
    return x, w


def qbx_workspace_bytes(n_src, n_ctr, ncoef, nrhs) -> int:
    return int(lib().qbx_workspace_bytes(n_src, n_ctr, ncoef, nrhs))


class Plan:
    """qbx_plan_create / qbx_plan_destroy."""

    def __init__(self, q_tgt=16, q_src=64, workspace_bytes=None, device=None, n_src=0, n_ctr=0,
                 ncoef=2, nrhs=1):
        self.device = torch.cuda.current_device() if device is None else int(device)
        if workspace_bytes is None:
            workspace_bytes = max(qbx_workspace_bytes(n_src, n_ctr, ncoef, nrhs), 1 << 20)
        self.q_tgt, self.q_src, self.workspace_bytes = q_tgt, q_src, int(workspace_bytes)
        h = ctypes.c_void_p()
        _check(lib().qbx_plan_create(ctypes.byref(h), self.device, q_tgt, q_src, self.workspace_bytes))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().qbx_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qbx_plan_set_timing(plan: Plan, on=True):
    _check(lib().qbx_plan_set_timing(plan.handle, 1 if on else 0))


def qbx_plan_set_min_waves(plan: Plan, waves: int):
    _check(lib().qbx_plan_set_min_waves(plan.handle, int(waves)))


def qbx_plan_kernel_ms(plan: Plan) -> float:
    """Device milliseconds of the pair-sum launches of the plan's last apply."""
    ms = ctypes.c_float(0.0)
    _check(lib().qbx_plan_kernel_ms(plan.handle, ctypes.byref(ms)))
    return float(ms.value)


def qbx_plan_create(q_tgt=16, q_src=64, workspace_bytes=None, device=None, **kw) -> Plan:
    return Plan(q_tgt, q_src, workspace_bytes, device, **kw)


def qbx_sync_status(plan: Plan):
    _check(lib().qbx_sync_status(plan.handle, _stream()))


class Geometry:
    """Device arrays of a discretised curve (qbx_geom) and the parameter values
    of the target / source nodes."""

    def __init__(self, M, q_tgt, q_src, device):
        f64 = dict(dtype=torch.float64, device=device)
        self.M, self.q_tgt, self.q_src = M, q_tgt, q_src
        self.n_tgt, self.n_src = M * q_tgt, M * q_src
        self.t = {}
        for n in ("src_x", "src_y", "src_nx", "src_ny", "src_w"):
            self.t[n] = torch.zeros(self.n_src, **f64)
        for n in ("tgt_x", "tgt_y", "tgt_nx", "tgt_ny", "tgt_w"):
            self.t[n] = torch.zeros(self.n_tgt, **f64)
        self.t["panel_h"] = torch.zeros(M, **f64)
        for n in ("ctr_x", "ctr_y", "ctr_r", "ctr_ratio"):
            self.t[n] = torch.zeros(2 * self.n_tgt, **f64)
        self.s = GeomStruct(M, q_tgt, q_src, self.n_tgt, self.n_src,
                            *[ctypes.c_void_p(self.t[n].data_ptr()) for n in (
                                "src_x", "src_y", "src_nx", "src_ny", "src_w",
                                "tgt_x", "tgt_y", "tgt_nx", "tgt_ny", "tgt_w",
                                "panel_h", "ctr_x", "ctr_y", "ctr_r", "ctr_ratio")])

    def __getitem__(self, name):
        return self.t[name]

    def ref(self):
        return ctypes.byref(self.s)


def panel_nodes(t_edges, q):
    """Curve parameter at the q-node GL points of each panel (library's GL rule)."""
    x, _ = qbx_gauss_legendre(q)
    t_edges = np.asarray(t_edges, dtype=np.float64)
    a, b = t_edges[:-1], t_edges[1:]
    return (0.5 * (a + b)[:, None] + 0.5 * (b - a)[:, None] * x[None, :]).reshape(-1)


RADIUS_H, RADIUS_SQRT_H, RADIUS_ADMISSIBLE = 0, 1, 2


def qbx_geometry(plan: Plan, curve, t_edges, r_factor=0.5, rule=RADIUS_H) -> Geometry:
    """Sample `curve` (t -> (gamma [n,2], gamma' [n,2])) at the panels' GL nodes
    and run qbx_geometry on the device."""
    dev = torch.device("cuda", plan.device)
    t_edges = np.asarray(t_edges, dtype=np.float64)
    t_tgt = panel_nodes(t_edges, plan.q_tgt)
    t_src = panel_nodes(t_edges, plan.q_src)
    gt, dgt = curve(t_tgt)
    gs, dgs = curve(t_src)
    up = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    return qbx_geometry_samples(plan, t_edges, up(gt), up(dgt), up(gs), up(dgs), r_factor, rule)


def qbx_geometry_samples(plan: Plan, t_edges, gam_tgt, dgam_tgt, gam_src, dgam_src, r_factor=0.5,
                         rule=RADIUS_H) -> Geometry:
    """qbx_geometry from curve samples already on the device: gamma, gamma' at
    the target nodes [n_tgt, 2] and at the source nodes [n_src, 2] (float64,
    at panel_nodes(t_edges, q) of the plan's grids)."""
    dev = torch.device("cuda", plan.device)
    t_edges = np.asarray(t_edges, dtype=np.float64)
    M = t_edges.size - 1
    g = Geometry(M, plan.q_tgt, plan.q_src, dev)
    arrs = [gam_tgt, dgam_tgt, gam_src, dgam_src]
    shapes = [(g.n_tgt, 2), (g.n_tgt, 2), (g.n_src, 2), (g.n_src, 2)]
    for a, shp in zip(arrs, shapes):
        if tuple(a.shape) != shp or a.dtype != torch.float64:
            raise ValueError(f"curve samples must be float64 of shape {shp}")
    g.inputs = [torch.as_tensor(t_edges, device=dev)] + [a.detach().contiguous() for a in arrs]
    g.r_factor = float(r_factor)
    g.t_tgt = panel_nodes(t_edges, plan.q_tgt)
    g.t_src = panel_nodes(t_edges, plan.q_src)
    _check(lib().qbx_geometry_rule(plan.handle, g.ref(), *[_ptr(a) for a in g.inputs], int(rule),
                                   float(r_factor), _stream()))
    g.rule = rule
    return g


def _dens2d(d, n):
    if d.dim() == 1:
        d = d.reshape(n, 1)
    if d.dtype != torch.complex128:
        raise TypeError("densities must be complex128")
    return d.contiguous()


def qbx_upsample(plan: Plan, g: Geometry, dens_tgt):
    d = _dens2d(dens_tgt, g.n_tgt)
    out = torch.empty((g.n_src, d.shape[1]), dtype=torch.complex128, device=d.device)
    _check(lib().qbx_upsample(plan.handle, g.ref(), _ptr(d), d.shape[1], _ptr(out), _stream()))
    return out


def _nctr(g, side):
    return 2 * g.n_tgt if side == SIDE_TWO else g.n_tgt


def qbx_form_locals(plan: Plan, g: Geometry, kind, side, k, p, wdens_src):
    wd = _dens2d(wdens_src, g.n_src)
    nrhs = wd.shape[1]
    alpha = torch.empty((_nctr(g, side), 2 * p + 1, nrhs), dtype=torch.complex128, device=wd.device)
    _check(lib().qbx_form_locals(plan.handle, g.ref(), kind, side, _k(k), p, _ptr(wd), nrhs,
                                 _ptr(alpha), _stream()))
    return alpha


def qbx_eval_locals(plan: Plan, g: Geometry, side, k, p, alpha, what=VALUE, ex=None, ey=None, ectr=None):
    nrhs = alpha.shape[2]
    if ex is None:
        n = 0
        n_out = _nctr(g, side)
    else:
        n = n_out = ex.numel()
    shape = (n_out, 2, nrhs) if what == GRAD else (n_out, nrhs)
    out = torch.empty(shape, dtype=torch.complex128, device=alpha.device)
    _check(lib().qbx_eval_locals(plan.handle, g.ref(), side, _k(k), p, _ptr(alpha.contiguous()), nrhs, what,
                                 n, _ptr(ex), _ptr(ey), _ptr(ectr), _ptr(out), _stream()))
    return out


def qbx_apply(plan: Plan, g: Geometry, op, side, limit, k, p, dens_tgt, x_far=None, out_on=None):
    """On-surface apply of S, D or grad S (plus far targets x_far [n,2])."""
    d = _dens2d(dens_tgt, g.n_tgt)
    nrhs = d.shape[1]
    shape = (g.n_tgt, 2, nrhs) if op in (OP_GRAD_S, OP_GRAD_D) else (g.n_tgt, nrhs)
    if out_on is None:
        out_on = torch.empty(shape, dtype=torch.complex128, device=d.device)
    n_far = 0 if x_far is None else x_far.shape[0]
    out_far = None
    if n_far:
        fshape = (n_far, 2, nrhs) if op == OP_GRAD_S else (n_far, nrhs)
        out_far = torch.empty(fshape, dtype=torch.complex128, device=d.device)
    _check(lib().qbx_apply(plan.handle, g.ref(), op, side, limit, _k(k), p, _ptr(d), nrhs, n_far,
                           _ptr(x_far.contiguous()) if n_far else None, _ptr(out_on), _ptr(out_far),
                           _stream()))
    return (out_on, out_far) if n_far else out_on


def qbx_apply_adjoint(plan: Plan, g: Geometry, op, side, limit, k, p, gout):
    """A^H gout for u = qbx_apply(..., op, ...) = A sigma (op S or D)."""
    go = _dens2d(gout, g.n_tgt)
    nrhs = go.shape[1]
    out = torch.empty_like(go)
    _check(lib().qbx_apply_adjoint(plan.handle, g.ref(), op, side, limit, _k(k), p, _ptr(go), nrhs, _ptr(out),
                                   _stream()))
    return out


class QBXApply(torch.autograd.Function):
    """u = A sigma through qbx_apply; backward = qbx_apply_adjoint (the
    transposed sweep), i.e. grad_sigma = A^H grad_u as torch's complex
    autograd expects for a complex-linear map."""

    @staticmethod
    def forward(ctx, dens, plan, g, op, side, limit, k, p):
        ctx.args = (plan, g, op, side, limit, k, p)
        return qbx_apply(plan, g, op, side, limit, k, p, dens.detach().contiguous())

    @staticmethod
    def backward(ctx, grad_u):
        plan, g, op, side, limit, k, p = ctx.args
        gd = qbx_apply_adjoint(plan, g, op, side, limit, k, p, grad_u.contiguous())
        return gd, None, None, None, None, None, None, None


def apply_autograd(plan: Plan, g: Geometry, op, side, limit, k, p, dens):
    """Differentiable on-surface apply of S or D (density gradients)."""
    return QBXApply.apply(dens, plan, g, op, side, limit, k, p)


def qbx_shape_adjoint_workspace_bytes(M, q_tgt, q_src, p, nrhs):
    return int(lib().qbx_shape_adjoint_workspace_bytes(M, q_tgt, q_src, p, nrhs))


def qbx_apply_shape_adjoint(plan: Plan, g: Geometry, side, k, p, dens, gout, op=OP_S):
    """Gradient of L = Re sum conj(gout) (S dens) (op = OP_S) or of
    Re sum conj(gout) (D dens) (op = OP_D) with respect to the curve samples
    given to qbx_geometry: returns (d gamma_tgt, d gamma'_tgt, d gamma_src,
    d gamma'_src), [n, 2] float64 each."""
    if op not in (OP_S, OP_D):
        raise ValueError("the shape adjoint covers S and D")
    if getattr(g, "rule", RADIUS_H) != RADIUS_H:
        raise ValueError("the shape adjoint needs r = r_factor * h (RADIUS_H)")
    d = _dens2d(dens, g.n_tgt)
    go = _dens2d(gout, g.n_tgt)
    if go.shape != d.shape:
        raise ValueError("gout and dens must have the same shape")
    f64 = dict(dtype=torch.float64, device=d.device)
    outs = [torch.empty((g.n_tgt, 2), **f64), torch.empty((g.n_tgt, 2), **f64),
            torch.empty((g.n_src, 2), **f64), torch.empty((g.n_src, 2), **f64)]
    dgt, dgs = g.inputs[2], g.inputs[4]
    fn = lib().qbx_apply_shape_adjoint if op == OP_S else lib().qbx_apply_shape_adjoint_d
    _check(fn(plan.handle, g.ref(), side, _k(k), p, _ptr(d), _ptr(go), d.shape[1], _ptr(dgt), _ptr(dgs),
              *[_ptr(o) for o in outs], _stream()))
    return tuple(outs)


class QBXShapeS(torch.autograd.Function):
    """u = S sigma on the curve given by its samples (gamma, gamma' at the
    target and source nodes): forward = qbx_geometry + qbx_apply; backward =
    qbx_apply_adjoint for sigma and qbx_apply_shape_adjoint for the samples."""

    @staticmethod
    def forward(ctx, dens, gam_tgt, dgam_tgt, gam_src, dgam_src, plan, t_edges, side, k, p, r_factor):
        g = qbx_geometry_samples(plan, t_edges, gam_tgt, dgam_tgt, gam_src, dgam_src, r_factor)
        d = dens.detach().contiguous()
        ctx.args = (plan, g, side, k, p, d)
        return qbx_apply(plan, g, OP_S, side, LIMIT_ONE_SIDED, k, p, d)

    @staticmethod
    def backward(ctx, grad_u):
        plan, g, side, k, p, d = ctx.args
        go = grad_u.contiguous()
        gd = qbx_apply_adjoint(plan, g, OP_S, side, LIMIT_ONE_SIDED, k, p, go) if ctx.needs_input_grad[0] else None
        shp = qbx_apply_shape_adjoint(plan, g, side, k, p, d, go) if any(ctx.needs_input_grad[1:5]) else (None,) * 4
        if gd is not None and gd.shape != grad_u.shape:
            gd = gd.reshape(grad_u.shape)
        return (gd,) + tuple(shp) + (None,) * 6


class QBXShapeD(torch.autograd.Function):
    """u = D mu (one-sided limit or PV) on the curve given by its samples:
    forward = qbx_geometry + qbx_apply; backward = qbx_apply_adjoint for mu
    and qbx_apply_shape_adjoint_d for the samples."""

    @staticmethod
    def forward(ctx, dens, gam_tgt, dgam_tgt, gam_src, dgam_src, plan, t_edges, side, limit, k, p, r_factor):
        g = qbx_geometry_samples(plan, t_edges, gam_tgt, dgam_tgt, gam_src, dgam_src, r_factor)
        d = dens.detach().contiguous()
        ctx.args = (plan, g, side, limit, k, p, d)
        return qbx_apply(plan, g, OP_D, side, limit, k, p, d)

    @staticmethod
    def backward(ctx, grad_u):
        plan, g, side, limit, k, p, d = ctx.args
        go = grad_u.contiguous()
        gd = qbx_apply_adjoint(plan, g, OP_D, side, limit, k, p, go) if ctx.needs_input_grad[0] else None
        shp = (qbx_apply_shape_adjoint(plan, g, side, k, p, d, go, op=OP_D) if any(ctx.needs_input_grad[1:5])
               else (None,) * 4)
        if gd is not None and gd.shape != grad_u.shape:
            gd = gd.reshape(grad_u.shape)
        return (gd,) + tuple(shp) + (None,) * 7


def apply_d_shape_autograd(plan: Plan, t_edges, gam_tgt, dgam_tgt, gam_src, dgam_src, dens, side, limit, k, p,
                           r_factor=0.5):
    """Differentiable D mu with respect to the density and to the curve samples."""
    return QBXShapeD.apply(dens, gam_tgt, dgam_tgt, gam_src, dgam_src, plan, t_edges, side, limit, k, p, r_factor)


def apply_s_shape_autograd(plan: Plan, t_edges, gam_tgt, dgam_tgt, gam_src, dgam_src, dens, side, k, p,
                           r_factor=0.5):
    """Differentiable S sigma with respect to the density and to the curve
    samples (for shape optimisation: build the samples in torch from the
    curve's parameters and let autograd carry the chain)."""
    return QBXShapeS.apply(dens, gam_tgt, dgam_tgt, gam_src, dgam_src, plan, t_edges, side, k, p, r_factor)


def qbx_assemble_cfie(plan: Plan, g: Geometry, k, eta, p):
    """The sqrt-weighted Nystrom matrix of 1/2 + D - i eta S (two-sided), as a
    [n][n] tensor holding A~ column-major: tensor[t', t] = A~[t, t']."""
    n = g.n_tgt
    A = torch.empty((n, n), dtype=torch.complex128, device=torch.device("cuda", plan.device))
    _check(lib().qbx_assemble_cfie(plan.handle, g.ref(), _k(k), _k(eta), p, _ptr(A), _stream()))
    return A


def qbx_solve_exterior_dirichlet(plan: Plan, g: Geometry, k, eta, p, f, tol=1e-10, restart=40, maxiter=200,
                                 mu0=None, raise_on_noconv=True, A=None):
    """GMRES for (1/2 + D - i eta S) mu = f (two-sided D and S, sqrt-weight
    unknowns).  Returns (mu, matvecs, relative residuals).  With A (from
    qbx_assemble_cfie with the same k, eta, p) every matvec is one complex
    matrix product (qbx_matmul_cm)."""
    ff = _dens2d(f, g.n_tgt)
    nrhs = ff.shape[1]
    mu = torch.zeros_like(ff) if mu0 is None else _dens2d(mu0, g.n_tgt).clone()
    it = ctypes.c_int(0)
    res = (ctypes.c_double * nrhs)()
    if A is None:
        rc = lib().qbx_solve_exterior_dirichlet(plan.handle, g.ref(), _k(k), _k(eta), p, _ptr(ff), nrhs, float(tol),
                                                restart, maxiter, _ptr(mu), ctypes.byref(it), res, _stream())
    else:
        rc = lib().qbx_solve_exterior_dirichlet_assembled(plan.handle, g.ref(), _ptr(A), _ptr(ff), nrhs, float(tol),
                                                          restart, maxiter, _ptr(mu), ctypes.byref(it), res,
                                                          _stream())
    if rc != 0 and (raise_on_noconv or rc != 5):
        _check(rc)
    return mu, it.value, np.array(res[:])


OPS_S, OPS_D, OPS_GRAD_S = 1, 2, 4


def qbx_matmul_cm(A, x, work=None):
    """y = A x for the column-major n x n matrix A (a tensor [n][n] holding
    A(i, j) at [j][i], the layout of qbx_assemble_cfie) and x [n][nrhs]
    (complex128 on the device), by the library's FP64 kernel."""
    n = A.shape[0]
    xx = _dens2d(x, n)
    nrhs = xx.shape[1]
    wb = lib().qbx_matmul_cm_work_bytes(n, nrhs)
    if work is None:
        work = torch.empty(max(wb, 16), dtype=torch.uint8, device=xx.device)
    y = torch.empty_like(xx)
    _check(lib().qbx_matmul_cm(n, nrhs, _ptr(A.contiguous()), _ptr(xx), _ptr(y), _ptr(work), work.numel(),
                               _stream()))
    return y


def qbx_vec_dots(V, w):
    """out[j][r] = sum_i conj(V[j][i][r]) w[i][r] for the Krylov vectors V
    [nv][n][nrhs] and w [n][nrhs] (complex128 on the device), in a fixed
    reduction order: the GMRES inner products, one per basis vector and
    right-hand side."""
    nv, n, nrhs = V.shape
    if tuple(w.shape) != (n, nrhs):
        raise ValueError("w must be [n][nrhs] like the rows of V")
    V, w = V.contiguous(), w.contiguous()
    work = torch.empty(int(lib().qbx_vec_dots_work_bytes(nrhs, nv)), dtype=torch.uint8, device=V.device)
    out = torch.empty((nv, nrhs), dtype=torch.complex128, device=V.device)
    _check(lib().qbx_vec_dots(n, nrhs, nv, _ptr(V), _ptr(w), _ptr(work), _ptr(out), _stream()))
    return out


def qbx_vec_orth_update(V, h, w):
    """w -= sum_j V[j] h[j] (per right-hand side), in place."""
    nv, n, nrhs = V.shape
    _check(lib().qbx_vec_orth_update(n, nrhs, nv, _ptr(V.contiguous()), _ptr(h.contiguous()), _ptr(w), _stream()))
    return w


def qbx_vec_combine(V, y, x):
    """x += sum_j V[j] y[j] (per right-hand side), in place."""
    nv, n, nrhs = V.shape
    _check(lib().qbx_vec_combine(n, nrhs, nv, _ptr(V.contiguous()), _ptr(y.contiguous()), _ptr(x), _stream()))
    return x


def qbx_apply_ops(plan: Plan, g: Geometry, ops, side, limit, k, p, dens, out=None, eta=None):
    """Several operators in one pass.  `ops`: iterable of OP_* codes; `dens`:
    one density tensor for all, or a dict {op: tensor}; returns {op: output}.
    eta > 0: near-only QBX (qbx_apply_local)."""
    ops = sorted(set(ops))
    if not isinstance(dens, dict):
        dens = {o: dens for o in ops}
    dd = {o: _dens2d(dens[o], g.n_tgt) for o in ops}
    nrhs = dd[ops[0]].shape[1]
    dev = dd[ops[0]].device
    if out is None:
        out = {}
    for o in ops:
        if o not in out:
            shape = (g.n_tgt, 2, nrhs) if o == OP_GRAD_S else (g.n_tgt, nrhs)
            out[o] = torch.empty(shape, dtype=torch.complex128, device=dev)
    dp = (_P * 3)(*[_ptr(dd[o]) if o in dd else None for o in range(3)])
    op_ = (_P * 3)(*[_ptr(out[o]) if o in out else None for o in range(3)])
    mask = sum(1 << o for o in ops)
    if eta is None:
        _check(lib().qbx_apply_ops(plan.handle, g.ref(), mask, side, limit, _k(k), p, dp, nrhs, op_, _stream()))
    else:
        _check(lib().qbx_apply_local(plan.handle, g.ref(), mask, side, limit, _k(k), p, float(eta), dp, nrhs, op_,
                                     _stream()))
    return {o: out[o] for o in ops}


def qbx_apply_cfie(plan: Plan, g: Geometry, k, eta, p, dens, out=None):
    """(D - i eta S) dens on both sides, the two kernel values of each pair
    combined before the rhs products (qbx_apply_cfie).  dens: [n_tgt] or
    [n_tgt][nrhs] complex128 device tensor; returns [n_tgt][nrhs]."""
    d = _dens2d(dens, g.n_tgt)
    nrhs = d.shape[1]
    if out is None:
        out = torch.empty((g.n_tgt, nrhs), dtype=torch.complex128, device=d.device)
    e = complex(eta)
    _check(lib().qbx_apply_cfie(plan.handle, g.ref(), _k(k), c64(e.real, e.imag), p, _ptr(d), nrhs, _ptr(out),
                                _stream()))
    return out


class Batch:
    """qbx_batch_create / qbx_batch_apply / qbx_batch_destroy: many curves in
    one persistent launch run as a CUDA graph.  `geoms`: Geometry objects made
    with `plan`; `ks`: wavenumbers; `dens`: per curve [n_tgt][nrhs] complex128
    device tensors, read at every apply; outputs are allocated here
    (self.out[i][op])."""

    def __init__(self, plan: Plan, geoms, ks, p, ops, side, limit, dens):
        n = len(geoms)
        self.plan, self.geoms = plan, list(geoms)
        self.dens = [_dens2d(d, g.n_tgt) for d, g in zip(dens, geoms)]
        nrhs = self.dens[0].shape[1]
        self.ops = sorted(set(ops))
        self.out = []
        for g, d in zip(self.geoms, self.dens):
            self.out.append({o: torch.empty((g.n_tgt, 2, nrhs) if o == OP_GRAD_S else (g.n_tgt, nrhs),
                                            dtype=torch.complex128, device=d.device) for o in self.ops})
        garr = (GeomStruct * n)(*[g.s for g in self.geoms])
        karr = (c64 * n)(*[_k(k) for k in ks])
        darr = (_P * n)(*[_ptr(d) for d in self.dens])
        oarr = (_P * (3 * n))(*[(_ptr(self.out[i][o]) if o in self.out[i] else None)
                                for i in range(n) for o in range(3)])
        mask = sum(1 << o for o in self.ops)
        h = ctypes.c_void_p()
        _check(lib().qbx_batch_create(ctypes.byref(h), plan.handle, n, garr, karr, p, mask, side, limit, nrhs,
                                      darr, oarr))
        self.handle = h

    def apply(self):
        _check(lib().qbx_batch_apply(self.handle, _stream()))
        return self.out

    def tune(self):
        """qbx_batch_tune: time the candidate configurations, keep the fastest."""
        rg, ch = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().qbx_batch_tune(self.handle, _stream(), ctypes.byref(rg), ctypes.byref(ch)))
        return rg.value, ch.value

    def set_eta(self, eta):
        """qbx_batch_set_eta: near-only QBX with this eta (> 0), or the global
        apply (0)."""
        _check(lib().qbx_batch_set_eta(self.handle, float(eta)))

    def info(self):
        """(rhs per warp group, sources per item, items, persistent CTAs)."""
        v = [ctypes.c_int(0) for _ in range(4)]
        _check(lib().qbx_batch_info(self.handle, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def status(self):
        _check(lib().qbx_batch_status(self.handle, _stream()))

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().qbx_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qbx_apply_static(g: Geometry, op, side, limit, k, p, dens_tgt, out_on=None):
    """On-surface apply without a plan: nothing is allocated by the library
    (scratch in a fixed device array, see include/qbx.h).  The output tensor is
    the caller's (allocated here by torch when out_on is None)."""
    d = _dens2d(dens_tgt, g.n_tgt)
    nrhs = d.shape[1]
    shape = (g.n_tgt, 2, nrhs) if op in (OP_GRAD_S, OP_GRAD_D) else (g.n_tgt, nrhs)
    if out_on is None:
        out_on = torch.empty(shape, dtype=torch.complex128, device=d.device)
    _check(lib().qbx_apply_static(g.ref(), op, side, limit, _k(k), p, _ptr(d), nrhs, _ptr(out_on), _stream()))
    return out_on


def qbx_apply_static_status():
    """Read and clear qbx_apply_static's device status word (raises
    QBXError(QBX_ENONFINITE) if a kernel produced a non-finite value)."""
    _check(lib().qbx_apply_static_status(_stream()))


def qbx_far(plan: Plan, g: Geometry, op, k, wdens_src, x_far):
    wd = _dens2d(wdens_src, g.n_src)
    nrhs = wd.shape[1]
    n = x_far.shape[0]
    shape = (n, 2, nrhs) if op == OP_GRAD_S else (n, nrhs)
    out = torch.empty(shape, dtype=torch.complex128, device=wd.device)
    _check(lib().qbx_far(plan.handle, g.ref(), op, _k(k), _ptr(wd), nrhs, n, _ptr(x_far.contiguous()),
                         _ptr(out), _stream()))
    return out


def qbx_assign_centres(plan: Plan, g: Geometry, side, xy):
    out = torch.empty(xy.shape[0], dtype=torch.int32, device=xy.device)
    _check(lib().qbx_assign_centres(plan.handle, g.ref(), side, xy.shape[0], _ptr(xy.contiguous()),
                                    _ptr(out), _stream()))
    return out


def qbx_debug_hankel01(z):
    z = z.to(torch.complex128).contiguous()
    h0 = torch.empty_like(z)
    h1 = torch.empty_like(z)
    _check(lib().qbx_debug_hankel01(_ptr(z), z.numel(), _ptr(h0), _ptr(h1), _stream()))
    return h0, h1


def qbx_debug_hankel01_ray(plan: Plan, k, rho):
    """(H0, H1) at z = k rho as the pair kernels evaluate them for this k
    (complex k: the plan's amplitude table of the ray where |z| >= 2)."""
    rho = rho.contiguous()
    h0 = torch.empty(rho.shape, dtype=torch.complex128, device=rho.device)
    h1 = torch.empty_like(h0)
    _check(lib().qbx_debug_hankel01_ray(plan.handle, _k(k), _ptr(rho), rho.numel(), _ptr(h0), _ptr(h1), _stream()))
    return h0, h1


def qbx_debug_besselj(z, nmax):
    z = z.to(torch.complex128).contiguous()
    out = torch.empty((z.numel(), nmax + 1), dtype=torch.complex128, device=z.device)
    _check(lib().qbx_debug_besselj(_ptr(z), z.numel(), nmax, _ptr(out), _stream()))
    return out
