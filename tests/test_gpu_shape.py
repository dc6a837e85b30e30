"""Shape adjoint of the on-surface S apply (reverse mode, GPU) against the
oracle's forward-mode shape derivative, and the shape-optimisation loss
||S sigma - g||^2 on the 128-panel starfish: gradient with respect to the 17
Fourier coefficients of r(t) by autograd, against central differences
(h = 1e-6) and against the oracle's derivative."""
import numpy as np
import pytest
import torch

import oracle
import paper_1207_4461_gb300 as qbx
import workloads as W

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def node_pert(seed, n_tgt, n_src):
    """A random direction for every sample (gamma, gamma' at every target and
    source node), as a callable of the node parameters (told apart by count)."""
    v = W.uniform(seed, 4 * (n_tgt + n_src)) - 0.5
    a, b = v[:2 * n_tgt].reshape(n_tgt, 2), v[2 * n_tgt:4 * n_tgt].reshape(n_tgt, 2)
    c = v[4 * n_tgt:4 * n_tgt + 2 * n_src].reshape(n_src, 2)
    d = v[4 * n_tgt + 2 * n_src:].reshape(n_src, 2)

    def fn(t):
        return (a, b) if np.asarray(t).size == n_tgt else (c, d)
    return fn


def fourier_pert(m, kind):
    def fn(t):
        t = np.asarray(t, dtype=np.float64)
        c, s = np.cos(t), np.sin(t)
        f = np.cos(m * t) if kind == "cos" else np.sin(m * t)
        df = -m * np.sin(m * t) if kind == "cos" else m * np.cos(m * t)
        return np.stack([f * c, f * s], -1), np.stack([df * c - f * s, df * s + f * c], -1)
    return fn


@pytest.mark.parametrize("side,k,nrhs,p", [(qbx.SIDE_INT, 5.0, 1, 8), (qbx.SIDE_EXT, 3 + 0.5j, 2, 8),
                                           (qbx.SIDE_TWO, 7.0, 3, 8), (qbx.SIDE_INT, 4.0, 1, 1),
                                           (qbx.SIDE_TWO, 2 + 0.3j, 2, 0)])
def test_shape_adjoint_vs_oracle_tangent(cuda, side, k, nrhs, p):
    """<grad, direction> from the reverse-mode GPU gradient equals the
    oracle's forward-mode Re sum conj(gout) du along random per-sample
    directions and Fourier directions: starfish, 12 panels (192 targets,
    768 sources), p = 8 and the edge orders p = 0, 1."""
    cur, M = W.starfish(), 12
    edges = cur.edges(M)
    n_t, n_s = M * 16, M * 64
    plan = qbx.Plan(16, 64, workspace_bytes=qbx.qbx_shape_adjoint_workspace_bytes(M, 16, 64, p, nrhs))
    g = qbx.qbx_geometry(plan, cur, edges)
    dens = W.complex_gaussian(11, n_t * nrhs).reshape(n_t, nrhs)
    gout = W.complex_gaussian(12, n_t * nrhs).reshape(n_t, nrhs)
    grads = [x.cpu().numpy() for x in qbx.qbx_apply_shape_adjoint(plan, g, side, k, p, dev(dens), dev(gout))]
    qbx.qbx_sync_status(plan)
    dirs = [node_pert(s, n_t, n_s) for s in (1, 2, 3)] + [fourier_pert(3, "cos"), fourier_pert(0, "cos"),
                                                         fourier_pert(2, "sin")]
    _, du = oracle.apply_s_tangent(cur, dirs, edges, 16, 64, side, k, p, dens)
    tt, ts = qbx.panel_nodes(edges, 16), qbx.panel_nodes(edges, 64)
    for j, d in enumerate(dirs):
        pt, pdt = d(tt)
        ps, pds = d(ts)
        gpu = (grads[0] * pt).sum() + (grads[1] * pdt).sum() + (grads[2] * ps).sum() + (grads[3] * pds).sum()
        ref = np.real(np.conj(gout) * du[j]).sum()
        scale = np.abs(gout * du[j]).sum()
        assert abs(gpu - ref) <= 1e-11 * scale, (j, gpu, ref, scale)


def test_shape_adjoint_translation_gradient_balances(cuda):
    """S is invariant under translations, so the gradients with respect to all
    sample positions sum to zero (the gamma' gradients need no balance)."""
    cur, M, p, k = W.starfish(), 16, 8, 6.0
    plan = qbx.Plan(16, 64, workspace_bytes=qbx.qbx_shape_adjoint_workspace_bytes(M, 16, 64, p, 1))
    g = qbx.qbx_geometry(plan, cur, cur.edges(M))
    dens = dev(W.density_cfg1(g.t_tgt).reshape(-1, 1))
    gout = dev(W.complex_gaussian(5, g.n_tgt).reshape(-1, 1))
    gt, _, gs, _ = qbx.qbx_apply_shape_adjoint(plan, g, qbx.SIDE_TWO, k, p, dens, gout)
    tot = (gt.sum(0) + gs.sum(0)).abs().max().item()
    scale = gt.abs().sum().item() + gs.abs().sum().item()
    assert tot <= 1e-13 * scale


def fourier_samples(coef, t, dev_):
    """gamma = r(t)(cos t, sin t), r = a0 + sum_{m=1..8} a_m cos mt + b_m sin mt,
    coef = (a0, a1..a8, b1..b8); gamma and gamma' at parameters t, in torch."""
    tt = torch.as_tensor(t, dtype=torch.float64, device=dev_)
    m = torch.arange(1, 9, dtype=torch.float64, device=dev_)
    cm, sm = torch.cos(tt[:, None] * m), torch.sin(tt[:, None] * m)
    a0, a, b = coef[0], coef[1:9], coef[9:17]
    r = a0 + cm @ a + sm @ b
    dr = (-sm * m) @ a + (cm * m) @ b
    c, s = torch.cos(tt), torch.sin(tt)
    gam = torch.stack([r * c, r * s], -1)
    dgam = torch.stack([dr * c - r * s, dr * s + r * c], -1)
    return gam, dgam


def test_starfish_128_fourier_gradient(cuda):
    """Loss ||S sigma - g||^2, g = e^{i k x.d}, d = (1, 0), on the starfish
    r = 1 + 0.25 cos 5t with 128 panels (2048 targets, 8192 sources), k = 10,
    p = 10, interior centres, sigma = cos 3t + 0.5 i sin t: the gradient with
    respect to the 17 Fourier coefficients of r by autograd through the shape
    adjoint, against central differences (h = 1e-6) of the GPU loss and
    against the oracle's forward-mode derivative; the density gradient of the
    same call against the density adjoint."""
    M, k, p = 128, 10.0, 10
    edges = np.linspace(0.0, 2 * np.pi, M + 1)
    plan = qbx.Plan(16, 64, workspace_bytes=qbx.qbx_shape_adjoint_workspace_bytes(M, 16, 64, p, 1))
    tt, ts = qbx.panel_nodes(edges, 16), qbx.panel_nodes(edges, 64)
    c0 = np.zeros(17)
    c0[0], c0[5] = 1.0, 0.25
    sig0 = dev(W.density_cfg1(tt).reshape(-1, 1))

    def loss(coef, sig):
        gt, dgt = fourier_samples(coef, tt, "cuda")
        gs, dgs = fourier_samples(coef, ts, "cuda")
        u = qbx.apply_s_shape_autograd(plan, edges, gt, dgt, gs, dgs, sig, qbx.SIDE_INT, k, p)
        target = torch.exp(1j * k * gt[:, 0]).reshape(-1, 1)
        return (torch.abs(u - target) ** 2).sum()

    coef = dev(c0).requires_grad_(True)
    sig = sig0.clone().requires_grad_(True)
    L = loss(coef, sig)
    L.backward()
    grad = coef.grad.detach().cpu().numpy()
    # central differences of the GPU loss
    h = 1e-6
    floor = 8 * 2.2e-16 * L.item() / h
    with torch.no_grad():
        for j in range(17):
            e = np.zeros(17)
            e[j] = h
            fd = (loss(dev(c0 + e), sig0) - loss(dev(c0 - e), sig0)).item() / (2 * h)
            assert abs(fd - grad[j]) <= floor + 1e-7 * abs(grad[j]), (j, fd, grad[j], floor)
    # the oracle's forward-mode derivative along each coefficient
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
    sg = W.density_cfg1(oracle.panel_nodes(edges, 16))
    u_o, du_o = oracle.apply_s_tangent(cur, dirs, edges, 16, 64, oracle.SIDE_INT, k, p, sg)
    go = oracle.geometry(cur, edges, 16, 64)
    tx = go["tgt_x"]
    tg = np.exp(1j * k * tx)
    res = u_o[:, 0] - tg
    ref = np.empty(17)
    for j, d in enumerate(dirs):
        dx = d(oracle.panel_nodes(edges, 16))[0][:, 0]
        ref[j] = 2.0 * np.real(np.conj(res) * (du_o[j][:, 0] - 1j * k * dx * tg)).sum()
    assert np.abs(grad - ref).max() <= 1e-9 * np.abs(ref).max(), (grad, ref)
    # density gradient: the same as the plain density adjoint
    g = qbx.qbx_geometry(plan, cur, edges)
    u = qbx.qbx_apply(plan, g, qbx.OP_S, qbx.SIDE_INT, 0, k, p, sig0)
    gd = qbx.qbx_apply_adjoint(plan, g, qbx.OP_S, qbx.SIDE_INT, 0, k, p,
                               2 * (u - torch.exp(1j * k * g["tgt_x"]).reshape(-1, 1)))
    assert (sig.grad - gd).abs().max().item() <= 1e-11 * gd.abs().max().item()


def test_shape_adjoint_errors(cuda):
    cur, M, p = W.starfish(), 8, 8
    plan = qbx.Plan(16, 64, workspace_bytes=1 << 12)
    g = qbx.qbx_geometry(plan, cur, cur.edges(M))
    d = dev(W.density_cfg1(g.t_tgt).reshape(-1, 1))
    with pytest.raises(qbx.QBXError) as e:
        qbx.qbx_apply_shape_adjoint(plan, g, qbx.SIDE_INT, 5.0, p, d, d)
    assert e.value.code == 7
    big = qbx.Plan(16, 64, workspace_bytes=qbx.qbx_shape_adjoint_workspace_bytes(M, 16, 64, p, 1))
    gb = qbx.qbx_geometry(big, cur, cur.edges(M))
    with pytest.raises(qbx.QBXError) as e:
        qbx.qbx_apply_shape_adjoint(big, gb, 5, 5.0, p, d, d)
    assert e.value.code == 1
    with pytest.raises(qbx.QBXError) as e:
        qbx.qbx_apply_shape_adjoint(big, gb, qbx.SIDE_INT, -1.0, p, d, d)
    assert e.value.code == 1
