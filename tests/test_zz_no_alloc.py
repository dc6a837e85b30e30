"""qbx_apply_static, the apply for callers that cannot allocate device memory
(memory owned by a pooling allocator, loops that cannot take cudaMalloc's
synchronisation): called through the C ABI, it must match the CPU oracle and
the plan-based entry point qbx_apply, keep calls in order on one stream
correct when they change the grid pair between them, report a non-finite
result through its status word, and refuse sizes beyond its fixed scratch.
This file is collected last so that a run stopping at the first failure has
already run every other test; its first test runs first in a fresh process,
so there the very first call is made on a non-blocking stream."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1207_4461_gb300 as qbx
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11
QBX_ENONFINITE = 4


def rel(a, b):
    a, b = (x.detach().cpu().numpy() if torch.is_tensor(x) else np.asarray(x) for x in (a, b))
    return np.abs(a - b).max() / np.abs(b).max()


def call_static(g, op, side, limit, k, p, dens, out, stream=None):
    """Direct C-ABI call (no binding logic in between) on `stream` (torch's
    current stream by default)."""
    L = qbx.lib()
    st = stream if stream is not None else torch.cuda.current_stream()
    return L.qbx_apply_static(g.ref(), op, side, limit, qbx.c64(complex(k).real, complex(k).imag), p,
                              ctypes.c_void_p(dens.data_ptr()), dens.shape[1],
                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream))


def static_status(stream=None):
    st = stream if stream is not None else torch.cuda.current_stream()
    return qbx.lib().qbx_apply_static_status(ctypes.c_void_p(st.cuda_stream))


def out_like(g, op, nrhs):
    shape = (g.n_tgt, 2, nrhs) if op == qbx.OP_GRAD_S else (g.n_tgt, nrhs)
    return torch.full(shape, complex(float("nan"), float("nan")), dtype=torch.complex128, device="cuda")


def geometry_pair(curve, M, q_tgt, q_src):
    plan = qbx.Plan(q_tgt, q_src, n_src=M * q_src, n_ctr=2 * M * q_tgt)
    g = qbx.qbx_geometry(plan, curve, curve.edges(M))
    go = oracle.geometry(curve, curve.edges(M), q_tgt, q_src)
    return plan, g, go


def test_static_apply_alternating_grid_pairs_on_one_stream(cuda):
    """Calls queued back to back on one non-blocking stream that switch between
    the (16, 64) and (8, 32) grid pairs (a new interpolation matrix each time)
    and between real and complex k (a new amplitude table): every result
    matches the oracle."""
    cur = W.starfish()
    nrhs = 2
    grids = {(16, 64): geometry_pair(cur, 20, 16, 64), (8, 32): geometry_pair(cur, 28, 8, 32)}
    calls = [((16, 64), qbx.OP_S, qbx.SIDE_INT, qbx.LIMIT_ONE_SIDED, 7.0, 9),
             ((8, 32), qbx.OP_D, qbx.SIDE_TWO, qbx.LIMIT_PV, 7.0, 8),
             ((16, 64), qbx.OP_GRAD_S, qbx.SIDE_EXT, qbx.LIMIT_PV, 4 + 0.5j, 9),
             ((8, 32), qbx.OP_S, qbx.SIDE_TWO, qbx.LIMIT_ONE_SIDED, 3 + 0.25j, 8)]
    dens = {key: W.complex_gaussian(31 + i, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
            for i, (key, (_, g, _)) in enumerate(grids.items())}
    dens_dev = {key: torch.as_tensor(d, device="cuda") for key, d in dens.items()}
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    outs = []
    with torch.cuda.stream(side):
        for key, op, sd, limit, k, p in calls:
            g = grids[key][1]
            out = out_like(g, op, nrhs)
            assert call_static(g, op, sd, limit, k, p, dens_dev[key], out, side) == 0, qbx.lib().qbx_last_error()
            outs.append(out)
        assert static_status(side) == 0
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    for (key, op, sd, limit, k, p), out in zip(calls, outs):
        go = grids[key][2]
        ref = oracle.apply(go, op, sd, limit, k, p, dens[key])
        assert rel(out, ref) < TOL, (key, op, k)


def test_static_apply_matches_oracle_and_plan_apply_twice(cuda):
    M, p, nrhs = 24, 10, 3
    plan = qbx.Plan(16, 64, n_src=M * 64, n_ctr=2 * M * 16, ncoef=2, nrhs=nrhs)
    cur = W.starfish()
    g = qbx.qbx_geometry(plan, cur, cur.edges(M))
    go = oracle.geometry(cur, cur.edges(M), 16, 64)
    dens_h = W.complex_gaussian(17, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    dens = torch.as_tensor(dens_h, device="cuda")
    calls = [(qbx.OP_D, qbx.SIDE_TWO, qbx.LIMIT_ONE_SIDED, 9.0),
             (qbx.OP_GRAD_S, qbx.SIDE_INT, qbx.LIMIT_PV, 4 + 0.5j)]
    for op, side, limit, k in calls:
        ref = qbx.qbx_apply(plan, g, op, side, limit, k, p, dens)
        out = out_like(g, op, nrhs)
        assert call_static(g, op, side, limit, k, p, dens, out) == 0, qbx.lib().qbx_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(out)).all()
        assert rel(out, ref) < TOL
        assert rel(out, oracle.apply(go, op, side, limit, k, p, dens_h)) < TOL
    # one rhs: the weighted-seed kernel instance, as qbx_apply takes it
    d1 = dens[:, :1].contiguous()
    out = out_like(g, qbx.OP_S, 1)
    assert call_static(g, qbx.OP_S, qbx.SIDE_EXT, qbx.LIMIT_ONE_SIDED, 9.0, p, d1, out) == 0
    torch.cuda.synchronize()
    assert rel(out, oracle.apply(go, qbx.OP_S, qbx.SIDE_EXT, 0, 9.0, p, dens_h[:, :1])) < TOL
    assert static_status() == 0


def test_static_apply_reports_non_finite_density(cuda):
    M, p = 8, 6
    plan, g, go = geometry_pair(W.circle(1.0), M, 16, 64)
    dens = torch.ones((g.n_tgt, 1), dtype=torch.complex128, device="cuda")
    dens[5, 0] = complex(float("nan"), 0.0)
    out = out_like(g, qbx.OP_S, 1)
    assert static_status() == 0
    assert call_static(g, qbx.OP_S, qbx.SIDE_INT, qbx.LIMIT_ONE_SIDED, 3.0, p, dens, out) == 0
    assert static_status() == QBX_ENONFINITE
    assert b"non-finite" in qbx.lib().qbx_last_error()
    # the read cleared the word: a clean call reports nothing
    dens[5, 0] = 1.0
    assert call_static(g, qbx.OP_S, qbx.SIDE_INT, qbx.LIMIT_ONE_SIDED, 3.0, p, dens, out) == 0
    assert static_status() == 0


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
