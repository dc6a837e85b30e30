"""qbx_apply_static, the apply for callers that cannot allocate device memory
(memory owned by a pooling allocator, loops that cannot take cudaMalloc's
synchronisation): called through the C ABI, it must reproduce qbx_apply, the
plan-based entry point, on two calls in a row, and refuse sizes beyond its
fixed scratch.  This file is collected last so that a run stopping at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1207_4461_gb300 as qbx
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11


def rel(a, b):
    return (torch.abs(a - b).max() / torch.abs(b).max()).item()


def call_static(g, op, side, limit, k, p, dens, out):
    """Direct C-ABI call (no binding logic in between)."""
    L = qbx.lib()
    rc = L.qbx_apply_static(g.ref(), op, side, limit, qbx.c64(complex(k).real, complex(k).imag), p,
                            ctypes.c_void_p(dens.data_ptr()), dens.shape[1],
                            ctypes.c_void_p(out.data_ptr()),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def test_static_apply_matches_plan_apply_twice(cuda):
    M, p, nrhs = 24, 10, 3
    plan = qbx.Plan(16, 64, n_src=M * 64, n_ctr=2 * M * 16, ncoef=2, nrhs=nrhs)
    cur = W.starfish()
    g = qbx.qbx_geometry(plan, cur, cur.edges(M))
    dens = torch.as_tensor(W.complex_gaussian(17, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs), device="cuda")
    calls = [(qbx.OP_D, qbx.SIDE_TWO, qbx.LIMIT_ONE_SIDED, 9.0),
             (qbx.OP_GRAD_S, qbx.SIDE_INT, qbx.LIMIT_PV, 4 + 0.5j)]
    for op, side, limit, k in calls:
        ref = qbx.qbx_apply(plan, g, op, side, limit, k, p, dens)
        out = torch.full_like(ref, complex(float("nan"), float("nan")))
        assert call_static(g, op, side, limit, k, p, dens, out) == 0, qbx.lib().qbx_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(out)).all()
        assert rel(out, ref) < TOL


def test_static_apply_rejects_sizes_beyond_its_scratch(cuda):
    M = 4
    plan = qbx.Plan(16, 64, n_src=M * 64, n_ctr=2 * M * 16)
    cur = W.circle(1.0)
    g = qbx.qbx_geometry(plan, cur, cur.edges(M))
    dens = torch.zeros((g.n_tgt, 1), dtype=torch.complex128, device="cuda")
    out = torch.zeros((g.n_tgt, 1), dtype=torch.complex128, device="cuda")
    # claim far more rhs than the 32 MiB scratch holds; rejected before any launch
    L = qbx.lib()
    rc = L.qbx_apply_static(g.ref(), qbx.OP_S, qbx.SIDE_INT, 0, qbx.c64(3.0, 0.0), 4,
                            ctypes.c_void_p(dens.data_ptr()), 1 << 20, ctypes.c_void_p(out.data_ptr()),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 7
    assert b"scratch" in L.qbx_last_error()
