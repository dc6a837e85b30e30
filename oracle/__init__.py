"""CPU FP64 oracle for QBX (quadrature by expansion), 2D Helmholtz.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The GPU library
(``paper_1207_4461_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``qbx_oracle.c`` (plain C99, compiled with gcc on
first use into ``oracle/_build/``); this module only marshals numpy arrays.
Each wrapper names the passage of Kloeckner, Barnett, Greengard, O'Neil,
"Quadrature by Expansion" (arXiv:1207.4461) that the C routine follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qbx_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libqbx_oracle.so")
_lock = threading.Lock()
_lib = None

OP_S, OP_D, OP_GRAD_S, OP_R, OP_GRAD_D = 0, 1, 2, 3, 4
SIDE_INT, SIDE_EXT, SIDE_TWO = 0, 1, 2
LIMIT_ONE_SIDED, LIMIT_PV = 0, 1


def build(force: bool = False) -> str:
    """Compile qbx_oracle.c into a shared library (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            L.orc_gauss_legendre.argtypes = [I, P, P]
            L.orc_hankel01_array.argtypes = [I, P, P, P]
            L.orc_hankel_seq_array.argtypes = [I, P, I, P]
            L.orc_besselj_seq_array.argtypes = [I, P, I, P]
            L.orc_geometry.argtypes = [I, I, I, P, P, P, P, P, D, I] + [P] * 15
            L.orc_upsample.argtypes = [I, I, I, I, P, P, P]
            L.orc_form_locals.argtypes = [I, I, P, P, I, P, P, P, P, P, I, D, D, I, P]
            L.orc_eval_locals.argtypes = [I, P, P, P, P, P, P, I, D, D, I, I, P]
            L.orc_apply.argtypes = [I, I, I, D, D, I, I, I, I] + [P] * 12 + [P, I, I, P, P]
            L.orc_far.argtypes = [I, I, P, I, P, P, P, P, P, I, D, D, P]
            L.orc_assign_centres.argtypes = [I, P, I, I, P, P, P, P]
            L.orc_apply_s_tangent.argtypes = [I, D, D, I, I, I, I, P, D] + [P] * 4 + [I] + [P] * 4 + [P, I, P, P]
            L.orc_apply_d_tangent.argtypes = [I, I, D, D, I, I, I, I, P, D] + [P] * 4 + [I] + [P] * 4 + [P, I, P, P]
            L.orc_apply_local.argtypes = [I, I, I, D, D, I, D, I, I, I] + [P] * 12 + [P, I, I, P, P]
            L.orc_num_threads.restype = I
            L.orc_set_num_threads.argtypes = [I]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ----------------------------------------------------------------------------
# Quadrature and special functions
# ----------------------------------------------------------------------------
def gauss_legendre(q: int):
    """q-node Gauss-Legendre rule on [-1, 1] (Newton on P_q), ascending nodes."""
    x = np.zeros(q)
    w = np.zeros(q)
    if lib().orc_gauss_legendre(q, _p(x), _p(w)) != 0:
        raise ValueError("bad q")
    return x, w


def hankel01(z):
    """H0^(1)(z), H1^(1)(z) for complex z, Im z >= 0 (the oracle's own series,
    Miller/Neumann and asymptotic routines)."""
    z = _c128(np.atleast_1d(z))
    h0 = np.zeros_like(z)
    h1 = np.zeros_like(z)
    lib().orc_hankel01_array(z.size, _p(z), _p(h0), _p(h1))
    return h0, h1


def hankel_seq(z, nmax: int):
    """H_0..H_nmax (upward recurrence), shape [len(z)][nmax+1]."""
    z = _c128(np.atleast_1d(z))
    out = np.zeros((z.size, nmax + 1), dtype=np.complex128)
    lib().orc_hankel_seq_array(z.size, _p(z), nmax, _p(out))
    return out


def besselj_seq(z, nmax: int):
    """J_0..J_nmax (ascending series for |z| <= 4, Miller otherwise)."""
    z = _c128(np.atleast_1d(z))
    out = np.zeros((z.size, nmax + 1), dtype=np.complex128)
    lib().orc_besselj_seq_array(z.size, _p(z), nmax, _p(out))
    return out


# ----------------------------------------------------------------------------
# Geometry / QBX
# ----------------------------------------------------------------------------
def panel_nodes(t_edges, q):
    """Parameter values of the q-node GL points of each panel (oracle's GL)."""
    x, _ = gauss_legendre(q)
    t_edges = np.asarray(t_edges, dtype=np.float64)
    a, b = t_edges[:-1], t_edges[1:]
    return (0.5 * (a + b)[:, None] + 0.5 * (b - a)[:, None] * x[None, :]).reshape(-1)


RADIUS_H, RADIUS_SQRT_H, RADIUS_ADMISSIBLE = 0, 1, 2


def geometry(curve, t_edges, q_tgt: int, q_src: int, r_factor: float = 0.5, rule: int = RADIUS_H):
    """Discretise `curve` (callable t -> (gamma [n,2], dgamma [n,2])) on panels
    with edges t_edges; Sec. 3.3 step 4a geometry and centres, with
    r = r_factor h (rule 0), r = r_factor sqrt(h) (rule 1, Sec. 3.1), or
    r = r_factor h lowered per centre to the largest radius whose disk holds
    no source node (rule 2, a departure from step 4a for sharp corners)."""
    t_edges = _f64(t_edges)
    M = t_edges.size - 1
    tt = panel_nodes(t_edges, q_tgt)
    ts = panel_nodes(t_edges, q_src)
    gt, dgt = (_f64(a) for a in curve(tt))
    gs, dgs = (_f64(a) for a in curve(ts))
    n_t, n_s = M * q_tgt, M * q_src
    g = {k: np.zeros(n_s) for k in ("src_x", "src_y", "src_nx", "src_ny", "src_w")}
    g.update({k: np.zeros(n_t) for k in ("tgt_x", "tgt_y", "tgt_nx", "tgt_ny", "tgt_w")})
    g["panel_h"] = np.zeros(M)
    g.update({k: np.zeros(2 * n_t) for k in ("ctr_x", "ctr_y", "ctr_r", "ctr_ratio")})
    rc = lib().orc_geometry(M, q_tgt, q_src, _p(t_edges), _p(gt), _p(dgt), _p(gs), _p(dgs),
                            float(r_factor), int(rule),
                            *[_p(g[k]) for k in ("src_x", "src_y", "src_nx", "src_ny", "src_w",
                                                 "tgt_x", "tgt_y", "tgt_nx", "tgt_ny", "tgt_w",
                                                 "panel_h", "ctr_x", "ctr_y", "ctr_r", "ctr_ratio")])
    if rc != 0:
        raise ValueError("orc_geometry failed")
    g.update(M=M, q_tgt=q_tgt, q_src=q_src, n_tgt=n_t, n_src=n_s, t_edges=t_edges,
             t_tgt=tt, t_src=ts)
    return g


def _dens2d(dens, n):
    d = _c128(dens)
    if d.ndim == 1:
        d = d.reshape(n, 1)
    return d


def upsample(g, dens_tgt):
    """Sec. 3.4.2: density on the target grid -> w_s * density on the source grid."""
    d = _dens2d(dens_tgt, g["n_tgt"])
    nrhs = d.shape[1]
    out = np.zeros((g["n_src"], nrhs), dtype=np.complex128)
    lib().orc_upsample(g["M"], g["q_tgt"], g["q_src"], nrhs, _p(g["src_w"]), _p(d), _p(out))
    return out


def _side_range(g, side):
    n = g["n_tgt"]
    return {SIDE_INT: (0, n), SIDE_EXT: (n, 2 * n), SIDE_TWO: (0, 2 * n)}[side]


def form_locals(g, kind, side, k, p, wdens):
    """Sec. 3.3 step 4b: alpha [n_ctr][2p+1][nrhs] for the centres of `side`."""
    wd = _dens2d(wdens, g["n_src"])
    nrhs = wd.shape[1]
    c0, c1 = _side_range(g, side)
    cx = _f64(g["ctr_x"][c0:c1])
    cy = _f64(g["ctr_y"][c0:c1])
    k = complex(k)
    alpha = np.zeros((c1 - c0, 2 * p + 1, nrhs), dtype=np.complex128)
    lib().orc_form_locals(kind, c1 - c0, _p(cx), _p(cy), g["n_src"], _p(g["src_x"]), _p(g["src_y"]),
                          _p(g["src_nx"]), _p(g["src_ny"]), _p(wd), nrhs, k.real, k.imag, p, _p(alpha))
    return alpha


def eval_locals(g, side, k, p, alpha, what=0, ex=None, ey=None, ectr=None):
    """Sec. 3.3 step 4c (and its gradient).  Default targets: each centre of
    `side` evaluated at its own on-surface target.  `ectr` indexes the centres
    of `side` (0-based within the side)."""
    c0, c1 = _side_range(g, side)
    cx = _f64(g["ctr_x"][c0:c1])
    cy = _f64(g["ctr_y"][c0:c1])
    alpha = _c128(alpha)
    nrhs = alpha.shape[2]
    if ex is None:
        nc = c1 - c0
        ex = _f64(np.concatenate([g["tgt_x"]] * (nc // g["n_tgt"])))
        ey = _f64(np.concatenate([g["tgt_y"]] * (nc // g["n_tgt"])))
        ectr = np.arange(nc, dtype=np.int32)
    ex, ey = _f64(ex), _f64(ey)
    ectr = np.ascontiguousarray(ectr, dtype=np.int32)
    n = ex.size
    k = complex(k)
    shape = (n, 2, nrhs) if what == 1 else (n, nrhs)
    out = np.zeros(shape, dtype=np.complex128)
    lib().orc_eval_locals(n, _p(ex), _p(ey), _p(ectr), _p(cx), _p(cy), _p(alpha), nrhs,
                          k.real, k.imag, p, what, _p(out))
    return out


def apply(g, op, side, limit, k, p, dens_tgt, sel=None):
    """Sec. 3.3 in full: one-sided limit, PV by jump subtraction, or two-sided
    average, of S, D or grad S at the on-surface targets (all, or the target
    indices `sel`, output row i for target sel[i])."""
    d = _dens2d(dens_tgt, g["n_tgt"])
    nrhs = d.shape[1]
    k = complex(k)
    if sel is None:
        n_out, n_sel, selp = g["n_tgt"], 0, None
    else:
        sel = np.ascontiguousarray(sel, dtype=np.int32)
        n_out, n_sel, selp = sel.size, sel.size, _p(sel)
    shape = (n_out, 2, nrhs) if op in (OP_GRAD_S, OP_GRAD_D) else (n_out, nrhs)
    out = np.zeros(shape, dtype=np.complex128)
    rc = lib().orc_apply(op, side, limit, k.real, k.imag, p, g["M"], g["q_tgt"], g["q_src"],
                         *[_p(g[n]) for n in ("src_x", "src_y", "src_nx", "src_ny", "src_w",
                                              "tgt_x", "tgt_y", "tgt_nx", "tgt_ny", "tgt_w",
                                              "ctr_x", "ctr_y")],
                         _p(d), nrhs, n_sel, selp, _p(out))
    if rc != 0:
        raise MemoryError("orc_apply failed")
    return out


def apply_local(g, op, side, limit, k, p, eta, dens_tgt, sel=None):
    """Near-only QBX (Sec. 5 remark): source nodes with |x_s - c| < eta r
    through the expansion at c, the rest by the smooth rule at the target;
    jumps as apply().  ops S, D, grad S; nrhs <= 64."""
    d = _dens2d(dens_tgt, g["n_tgt"])
    nrhs = d.shape[1]
    k = complex(k)
    if sel is None:
        n_out, n_sel, selp = g["n_tgt"], 0, None
    else:
        sel = np.ascontiguousarray(sel, dtype=np.int32)
        n_out, n_sel, selp = sel.size, sel.size, _p(sel)
    shape = (n_out, 2, nrhs) if op == OP_GRAD_S else (n_out, nrhs)
    out = np.zeros(shape, dtype=np.complex128)
    rc = lib().orc_apply_local(op, side, limit, k.real, k.imag, p, float(eta), g["M"], g["q_tgt"], g["q_src"],
                               *[_p(g[n]) for n in ("src_x", "src_y", "src_nx", "src_ny", "src_w",
                                                    "tgt_x", "tgt_y", "tgt_nx", "tgt_ny",
                                                    "ctr_x", "ctr_y", "ctr_r")],
                               _p(d), nrhs, n_sel, selp, _p(out))
    if rc != 0:
        raise ValueError(f"orc_apply_local failed ({rc})")
    return out


def matrix(g, op, side, limit, k, p):
    """The discrete operator as a matrix: column j is apply() of the j-th unit
    density (all columns at once, as nrhs = n_tgt right-hand sides).  Shape
    [n_tgt][n_tgt] for S and D, [n_tgt][2][n_tgt] for grad S.  For small
    problems: the adjoint of the apply is then conj(A).T."""
    n = g["n_tgt"]
    return apply(g, op, side, limit, k, p, np.eye(n, dtype=np.complex128))


def far(g, op, k, wdens, xy):
    """Plain smooth quadrature of S, D or grad S at off-surface points xy [n,2]."""
    wd = _dens2d(wdens, g["n_src"])
    nrhs = wd.shape[1]
    xy = _f64(np.asarray(xy).reshape(-1, 2))
    n = xy.shape[0]
    k = complex(k)
    shape = (n, 2, nrhs) if op == OP_GRAD_S else (n, nrhs)
    out = np.zeros(shape, dtype=np.complex128)
    lib().orc_far(op, n, _p(xy), g["n_src"], _p(g["src_x"]), _p(g["src_y"]), _p(g["src_nx"]),
                  _p(g["src_ny"]), _p(wd), nrhs, k.real, k.imag, _p(out))
    return out


def assign_centres(g, side, xy):
    """Centre (global index in [0, 2 n_tgt)) serving each off-surface point, or -1."""
    xy = _f64(np.asarray(xy).reshape(-1, 2))
    c0, c1 = _side_range(g, side)
    out = np.zeros(xy.shape[0], dtype=np.int32)
    lib().orc_assign_centres(xy.shape[0], _p(xy), c0, c1, _p(g["ctr_x"]), _p(g["ctr_y"]),
                             _p(g["ctr_r"]), _p(out))
    return out


def apply_s_tangent(curve, pert, t_edges, q_tgt: int, q_src: int, side, k, p, dens_tgt, r_factor: float = 0.5):
    """Shape derivative of the on-surface S apply, forward mode: with the curve
    samples moving along `pert` (callable t -> (d gamma [n,2], d gamma' [n,2]),
    or a list of such directions) and the density fixed on the target grid as
    a function of t, returns (u, du/d eps): u [n_tgt][nrhs], du the same shape
    (one direction) or [ndir][n_tgt][nrhs] (a list).  Geometry of Sec. 3.3
    step 4a and the sums of eqs. graf-coefficient / local-exp differentiated
    by the chain rule."""
    t_edges = _f64(t_edges)
    M = t_edges.size - 1
    tt = panel_nodes(t_edges, q_tgt)
    ts = panel_nodes(t_edges, q_src)
    gt, dgt = (_f64(a) for a in curve(tt))
    gs, dgs = (_f64(a) for a in curve(ts))
    perts = list(pert) if isinstance(pert, (list, tuple)) else [pert]
    nd = len(perts)
    pgt = _f64(np.stack([_f64(q(tt)[0]) for q in perts]))
    pdgt = _f64(np.stack([_f64(q(tt)[1]) for q in perts]))
    pgs = _f64(np.stack([_f64(q(ts)[0]) for q in perts]))
    pdgs = _f64(np.stack([_f64(q(ts)[1]) for q in perts]))
    d = _dens2d(dens_tgt, M * q_tgt)
    nrhs = d.shape[1]
    k = complex(k)
    u = np.zeros((M * q_tgt, nrhs), dtype=np.complex128)
    du = np.zeros((nd, M * q_tgt, nrhs), dtype=np.complex128)
    rc = lib().orc_apply_s_tangent(side, k.real, k.imag, p, M, q_tgt, q_src, _p(t_edges), float(r_factor),
                                   _p(gt), _p(dgt), _p(gs), _p(dgs), nd, _p(pgt), _p(pdgt), _p(pgs), _p(pdgs),
                                   _p(d), nrhs, _p(u), _p(du))
    if rc != 0:
        raise ValueError(f"orc_apply_s_tangent failed ({rc})")
    return u, (du if isinstance(pert, (list, tuple)) else du[0])


def apply_d_tangent(curve, pert, t_edges, q_tgt: int, q_src: int, side, limit, k, p, dens_tgt,
                    r_factor: float = 0.5):
    """Shape derivative of the on-surface D apply (limit ONE_SIDED or PV),
    forward mode, as apply_s_tangent: the D coefficients (eq.
    graf-coefficient-dlp) differentiated through the source positions,
    normals and weights and the centres; the PV jump does not move."""
    t_edges = _f64(t_edges)
    M = t_edges.size - 1
    tt = panel_nodes(t_edges, q_tgt)
    ts = panel_nodes(t_edges, q_src)
    gt, dgt = (_f64(a) for a in curve(tt))
    gs, dgs = (_f64(a) for a in curve(ts))
    perts = list(pert) if isinstance(pert, (list, tuple)) else [pert]
    nd = len(perts)
    pgt = _f64(np.stack([_f64(q(tt)[0]) for q in perts]))
    pdgt = _f64(np.stack([_f64(q(tt)[1]) for q in perts]))
    pgs = _f64(np.stack([_f64(q(ts)[0]) for q in perts]))
    pdgs = _f64(np.stack([_f64(q(ts)[1]) for q in perts]))
    d = _dens2d(dens_tgt, M * q_tgt)
    nrhs = d.shape[1]
    k = complex(k)
    u = np.zeros((M * q_tgt, nrhs), dtype=np.complex128)
    du = np.zeros((nd, M * q_tgt, nrhs), dtype=np.complex128)
    rc = lib().orc_apply_d_tangent(side, limit, k.real, k.imag, p, M, q_tgt, q_src, _p(t_edges), float(r_factor),
                                   _p(gt), _p(dgt), _p(gs), _p(dgs), nd, _p(pgt), _p(pdgt), _p(pgs), _p(pdgs),
                                   _p(d), nrhs, _p(u), _p(du))
    if rc != 0:
        raise ValueError(f"orc_apply_d_tangent failed ({rc})")
    return u, (du if isinstance(pert, (list, tuple)) else du[0])


def set_num_threads(n: int):
    """OpenMP threads of the oracle's parallel loops (results do not depend on it)."""
    lib().orc_set_num_threads(int(n))
