"""The adjoint (transposed sweep) of the on-surface apply with respect to the
density: against the oracle's operator matrix, the inner-product identity at
the 128-panel size, and torch autograd against central finite differences."""
import numpy as np
import pytest
import torch

import oracle
import paper_1207_4461_gb300 as qbx
import workloads as W

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("op", [qbx.OP_S, qbx.OP_D])
@pytest.mark.parametrize("side,limit,k,nrhs", [(qbx.SIDE_INT, 0, 5.0, 1), (qbx.SIDE_EXT, 1, 3 + 0.5j, 3),
                                               (qbx.SIDE_TWO, 0, 9.0, 12), (qbx.SIDE_INT, 1, 7.0, 2)])
def test_adjoint_matches_oracle_matrix(cuda, op, side, limit, k, nrhs):
    """A^H g with A the oracle's operator matrix (column j = apply of the j-th
    unit density): 5 panels, 80 targets (2.5 tiles), 320 sources."""
    M, p = 5, 7
    cur = W.starfish(0.2, 3)
    plan = qbx.Plan(16, 64, n_src=M * 64, n_ctr=2 * M * 16, ncoef=2 * p + 1, nrhs=nrhs)
    g = qbx.qbx_geometry(plan, cur, cur.edges(M))
    go = oracle.geometry(cur, cur.edges(M), 16, 64)
    A = oracle.matrix(go, op, side, limit, k, p)
    gout = W.complex_gaussian(123, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    ref = A.conj().T @ gout
    got = qbx.qbx_apply_adjoint(plan, g, op, side, limit, k, p, dev(gout)).cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-11
    qbx.qbx_sync_status(plan)


@pytest.mark.parametrize("op", [qbx.OP_S, qbx.OP_D])
def test_adjoint_inner_product_identity_128_panels(cuda, op):
    """<A s, g> = <s, A^H g> on the starfish with 128 panels (2048 targets,
    8192 sources), k = 10, p = 10, interior centres."""
    M, k, p, nrhs = 128, 10.0, 10, 2
    cur = W.starfish()
    plan = qbx.Plan(16, 64, n_src=M * 64, n_ctr=2 * M * 16, ncoef=2, nrhs=nrhs)
    g = qbx.qbx_geometry(plan, cur, cur.edges(M))
    s = dev(W.complex_gaussian(1, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs))
    gg = dev(W.complex_gaussian(2, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs))
    As = qbx.qbx_apply(plan, g, op, qbx.SIDE_INT, qbx.LIMIT_PV, k, p, s)
    Ahg = qbx.qbx_apply_adjoint(plan, g, op, qbx.SIDE_INT, qbx.LIMIT_PV, k, p, gg)
    lhs = (As.conj() * gg).sum(0)
    rhs = (s.conj() * Ahg).sum(0)
    scale = (torch.abs(As) * torch.abs(gg)).sum(0)
    assert (torch.abs(lhs - rhs) / scale).max().item() < 1e-13


def test_autograd_loss_gradient_vs_central_differences(cuda):
    """L(sigma) = ||S sigma - g||^2, g = e^{i k x.d}, d = (1, 0), on the
    starfish with 128 panels, k = 10, p = 10 (interior): torch autograd through
    the adjoint against central differences (h = 1e-6) in Re and Im of
    several density values.  L is quadratic, so the central difference is
    exact up to rounding."""
    M, k, p = 128, 10.0, 10
    cur = W.starfish()
    plan = qbx.Plan(16, 64, n_src=M * 64, n_ctr=2 * M * 16, ncoef=2, nrhs=1)
    g = qbx.qbx_geometry(plan, cur, cur.edges(M))
    target = torch.exp(1j * k * g["tgt_x"]).reshape(-1, 1)
    sigma0 = dev(W.density_cfg1(g.t_tgt).reshape(-1, 1))

    def loss(sig):
        u = qbx.apply_autograd(plan, g, qbx.OP_S, qbx.SIDE_INT, 0, k, p, sig)
        return (torch.abs(u - target) ** 2).sum()

    sig = sigma0.clone().requires_grad_(True)
    L = loss(sig)
    L.backward()
    grad = sig.grad.detach()
    h = 1e-6
    # rounding floor of a central difference of L: a few eps * L / h
    floor = 8 * 2.2e-16 * L.item() / h
    for j in (0, 17, 1000, 2047):
        for unit in (1.0, 1j):
            e = torch.zeros_like(sigma0)
            e[j, 0] = unit * h
            fd = (loss(sigma0 + e) - loss(sigma0 - e)).item() / (2 * h)
            # torch's convention: grad = dL/dRe + i dL/dIm
            an = grad[j, 0].real.item() if unit == 1.0 else grad[j, 0].imag.item()
            assert abs(fd - an) <= floor + 1e-8 * abs(an), (j, unit, fd, an, floor)


@pytest.mark.parametrize("seed", range(8))
def test_random_adjoint_inner_product(cuda, seed):
    """Seeded random cases: operator S or D, side, limit, real or complex k,
    order, rhs count (1-20), panel count: <A s, g> = <s, A^H g> with the
    forward apply and the transposed sweep of the library, and A^H g against
    the oracle's operator matrix at the smaller sizes."""
    rng = np.random.default_rng(500 + seed)
    op = (qbx.OP_S, qbx.OP_D)[seed % 2]
    side = (qbx.SIDE_INT, qbx.SIDE_EXT, qbx.SIDE_TWO)[int(rng.integers(3))]
    limit = int(rng.integers(2))
    kr = float(rng.uniform(1.0, 12.0))
    k = complex(kr, float(rng.uniform(0.05, 1.0))) if rng.random() < 0.5 else kr
    p = int(rng.integers(1, 11))
    nrhs = int(rng.choice([1, 2, 5, 20]))
    M = int(rng.integers(4, 9))
    cur = W.starfish(0.2, 3)
    plan = qbx.Plan(16, 64, n_src=M * 64, n_ctr=2 * M * 16, ncoef=2 * p + 1, nrhs=nrhs)
    g = qbx.qbx_geometry(plan, cur, cur.edges(M))
    s = W.complex_gaussian(seed + 1, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    gg = W.complex_gaussian(seed + 2, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    As = qbx.qbx_apply(plan, g, op, side, limit, k, p, dev(s))
    Ahg = qbx.qbx_apply_adjoint(plan, g, op, side, limit, k, p, dev(gg))
    qbx.qbx_sync_status(plan)
    lhs = (As.conj() * dev(gg)).sum(0)
    rhs = (dev(s).conj() * Ahg).sum(0)
    scale = (torch.abs(As) * torch.abs(dev(gg))).sum(0)
    assert (torch.abs(lhs - rhs) / scale).max().item() < 1e-13, (op, side, limit, k, p, nrhs, M)
    go = oracle.geometry(cur, cur.edges(M), 16, 64)
    A = oracle.matrix(go, op, side, limit, k, p)
    ref = A.conj().T @ gg
    assert np.abs(Ahg.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-11, (op, side, limit, k, p, nrhs, M)
