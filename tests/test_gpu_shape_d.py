"""Shape adjoint of the on-surface D apply (reverse mode, GPU: second source
derivatives of the Graf sum, the source normals, weights and centres)
against the oracle's forward-mode shape derivative of D, and a loss on the
128-panel starfish differentiated with respect to the 17 Fourier
coefficients of r(t) by autograd, against central differences (h = 1e-6)
and the oracle's derivative."""
import numpy as np
import pytest
import torch

import oracle
import paper_1207_4461_gb300 as qbx
import workloads as W
from test_gpu_shape import dev, fourier_pert, fourier_samples, node_pert

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("side,limit,k,nrhs,p", [(qbx.SIDE_INT, qbx.LIMIT_ONE_SIDED, 5.0, 1, 8),
                                                 (qbx.SIDE_EXT, qbx.LIMIT_PV, 3 + 0.5j, 2, 8),
                                                 (qbx.SIDE_TWO, qbx.LIMIT_ONE_SIDED, 7.0, 5, 8),
                                                 (qbx.SIDE_INT, qbx.LIMIT_PV, 4.0, 1, 0),
                                                 (qbx.SIDE_TWO, qbx.LIMIT_ONE_SIDED, 2 + 0.3j, 2, 1)])
def test_shape_adjoint_d_vs_oracle_tangent(cuda, side, limit, k, nrhs, p):
    """<grad, direction> from the reverse-mode GPU gradient of
    Re sum conj(gout) D mu equals the oracle's forward-mode derivative along
    random per-sample directions and Fourier directions: starfish, 12 panels
    (192 targets, 768 sources), p = 8, and the edge orders p = 0, 1 (where the
    sums by parts reduce to their end terms); 5 rhs take two passes of 4."""
    cur, M = W.starfish(), 12
    edges = cur.edges(M)
    n_t, n_s = M * 16, M * 64
    plan = qbx.Plan(16, 64, workspace_bytes=qbx.qbx_shape_adjoint_workspace_bytes(M, 16, 64, p, nrhs))
    g = qbx.qbx_geometry(plan, cur, edges)
    dens = W.complex_gaussian(21, n_t * nrhs).reshape(n_t, nrhs)
    gout = W.complex_gaussian(22, n_t * nrhs).reshape(n_t, nrhs)
    grads = [x.cpu().numpy() for x in qbx.qbx_apply_shape_adjoint(plan, g, side, k, p, dev(dens), dev(gout),
                                                                   op=qbx.OP_D)]
    qbx.qbx_sync_status(plan)
    dirs = [node_pert(s, n_t, n_s) for s in (4, 5, 6)] + [fourier_pert(3, "cos"), fourier_pert(0, "cos"),
                                                         fourier_pert(2, "sin")]
    _, du = oracle.apply_d_tangent(cur, dirs, edges, 16, 64, side, limit, k, p, dens)
    tt, ts = qbx.panel_nodes(edges, 16), qbx.panel_nodes(edges, 64)
    for j, d in enumerate(dirs):
        pt, pdt = d(tt)
        ps, pds = d(ts)
        gpu = (grads[0] * pt).sum() + (grads[1] * pdt).sum() + (grads[2] * ps).sum() + (grads[3] * pds).sum()
        ref = np.real(np.conj(gout) * du[j]).sum()
        scale = np.abs(gout * du[j]).sum()
        assert abs(gpu - ref) <= 1e-11 * scale, (j, gpu, ref, scale)


def test_shape_adjoint_d_rigid_motions(cuda):
    """D is invariant under translations and rotations of the curve: the
    position gradients sum to zero, and the gradient along an infinitesimal
    rotation (gamma -> R gamma, gamma' -> R gamma') vanishes."""
    cur, M, p, k = W.starfish(), 16, 8, 6.0
    plan = qbx.Plan(16, 64, workspace_bytes=qbx.qbx_shape_adjoint_workspace_bytes(M, 16, 64, p, 1))
    g = qbx.qbx_geometry(plan, cur, cur.edges(M))
    dens = dev(W.density_cfg1(g.t_tgt).reshape(-1, 1))
    gout = dev(W.complex_gaussian(5, g.n_tgt).reshape(-1, 1))
    gt, gdt, gs, gds = qbx.qbx_apply_shape_adjoint(plan, g, qbx.SIDE_TWO, k, p, dens, gout, op=qbx.OP_D)
    scale = gt.abs().sum().item() + gs.abs().sum().item()
    assert (gt.sum(0) + gs.sum(0)).abs().max().item() <= 1e-13 * scale
    rot = lambda v: torch.stack([-v[:, 1], v[:, 0]], 1)   # d/d angle of R(angle) v at 0
    xt, xs = torch.stack([g["tgt_x"], g["tgt_y"]], 1), torch.stack([g["src_x"], g["src_y"]], 1)
    dgt, dgs = g.inputs[2], g.inputs[4]
    dL = ((gt * rot(xt)).sum() + (gdt * rot(dgt)).sum() + (gs * rot(xs)).sum() + (gds * rot(dgs)).sum()).item()
    mag = ((gt * rot(xt)).abs().sum() + (gdt * rot(dgt)).abs().sum() + (gs * rot(xs)).abs().sum()
           + (gds * rot(dgs)).abs().sum()).item()
    assert abs(dL) <= 1e-12 * mag


def test_starfish_128_fourier_gradient_d(cuda):
    """Loss ||D mu - g||^2 (interior limit), g = e^{i k x.d}, d = (1, 0), on the
    starfish r = 1 + 0.25 cos 5t with 128 panels (2048 targets, 8192 sources),
    k = 10, p = 10, mu = cos 3t + 0.5 i sin t: the gradient with respect to
    the 17 Fourier coefficients of r by autograd through the D shape adjoint,
    against central differences (h = 1e-6) of the GPU loss and against the
    oracle's forward-mode derivative."""
    M, k, p = 128, 10.0, 10
    edges = np.linspace(0.0, 2 * np.pi, M + 1)
    plan = qbx.Plan(16, 64, workspace_bytes=qbx.qbx_shape_adjoint_workspace_bytes(M, 16, 64, p, 1))
    tt, ts = qbx.panel_nodes(edges, 16), qbx.panel_nodes(edges, 64)
    c0 = np.zeros(17)
    c0[0], c0[5] = 1.0, 0.25
    mu0 = dev(W.density_cfg1(tt).reshape(-1, 1))

    def loss(coef, mu):
        gt, dgt = fourier_samples(coef, tt, "cuda")
        gs, dgs = fourier_samples(coef, ts, "cuda")
        u = qbx.apply_d_shape_autograd(plan, edges, gt, dgt, gs, dgs, mu, qbx.SIDE_INT, qbx.LIMIT_ONE_SIDED, k, p)
        target = torch.exp(1j * k * gt[:, 0]).reshape(-1, 1)
        return (torch.abs(u - target) ** 2).sum()

    coef = dev(c0).requires_grad_(True)
    mu = mu0.clone().requires_grad_(True)
    L = loss(coef, mu)
    L.backward()
    grad = coef.grad.detach().cpu().numpy()
    h = 1e-6
    floor = 8 * 2.2e-16 * L.item() / h
    with torch.no_grad():
        for j in range(17):
            e = np.zeros(17)
            e[j] = h
            fd = (loss(dev(c0 + e), mu0) - loss(dev(c0 - e), mu0)).item() / (2 * h)
            assert abs(fd - grad[j]) <= floor + 1e-7 * abs(grad[j]), (j, fd, grad[j], floor)
    cur = W.starfish()

    def coef_dir(j):
        def fn(t):
            t = np.asarray(t, dtype=np.float64)
            if j == 0:
                f, df = np.ones_like(t), np.zeros_like(t)
            elif j <= 8:
                f, df = np.cos(j * t), -j * np.sin(j * t)
            else:
                m = j - 8
                f, df = np.sin(m * t), m * np.cos(m * t)
            c, s = np.cos(t), np.sin(t)
            return np.stack([f * c, f * s], -1), np.stack([df * c - f * s, df * s + f * c], -1)
        return fn
    dirs = [coef_dir(j) for j in range(17)]
    mg = W.density_cfg1(oracle.panel_nodes(edges, 16))
    u_o, du_o = oracle.apply_d_tangent(cur, dirs, edges, 16, 64, oracle.SIDE_INT, oracle.LIMIT_ONE_SIDED, k, p, mg)
    tx = oracle.geometry(cur, edges, 16, 64)["tgt_x"]
    tg = np.exp(1j * k * tx)
    res = u_o[:, 0] - tg
    ref = np.empty(17)
    for j, d in enumerate(dirs):
        dx = d(oracle.panel_nodes(edges, 16))[0][:, 0]
        ref[j] = 2.0 * np.real(np.conj(res) * (du_o[j][:, 0] - 1j * k * dx * tg)).sum()
    assert np.abs(grad - ref).max() <= 1e-9 * np.abs(ref).max(), (grad, ref)
    # density gradient: the same as the plain density adjoint
    g = qbx.qbx_geometry(plan, cur, edges)
    u = qbx.qbx_apply(plan, g, qbx.OP_D, qbx.SIDE_INT, 0, k, p, mu0)
    gd = qbx.qbx_apply_adjoint(plan, g, qbx.OP_D, qbx.SIDE_INT, 0, k, p,
                               2 * (u - torch.exp(1j * k * g["tgt_x"]).reshape(-1, 1)))
    assert (mu.grad - gd).abs().max().item() <= 1e-11 * gd.abs().max().item()
