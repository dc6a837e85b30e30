"""GPU parity: every step of the CUDA path against the CPU oracle, through the
C ABI, on the same seeded inputs.

Bar (A10 reading of the target): max-norm relative error
||u_gpu - u_oracle||_inf / ||u_oracle||_inf <= 1e-11 per output array;
integer outputs bit-exact.  Sizes span several CTA tiles (128 centres, 128
sources) with ragged tails; the full-size starfish (256 panels, k = 20,
p = 12, both sides) is checked on sampled targets.
"""
import math

import numpy as np
import pytest
import scipy.special as sp
import torch

import oracle
import paper_1207_4461_gb300 as qbx
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11


def rel(a, b):
    a = a.detach().cpu().numpy() if torch.is_tensor(a) else np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).max() / np.abs(b).max()


def make(curve, M, q_tgt=16, q_src=64, nrhs=1, p=12, extra_ctr=1):
    plan = qbx.Plan(q_tgt, q_src, n_src=M * q_src, n_ctr=2 * M * q_tgt * extra_ctr,
                    ncoef=max(2, 2 * p + 1), nrhs=nrhs)
    g = qbx.qbx_geometry(plan, curve, curve.edges(M))
    go = oracle.geometry(curve, curve.edges(M), q_tgt, q_src)
    return plan, g, go


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


# ---------------------------------------------------------------------------
# special functions (a2, a5) against scipy
# ---------------------------------------------------------------------------
def test_device_hankel_real(cuda):
    # dense grid, the series / fit switch at z = 2, and the fit interval edges z = 64/i
    z = np.concatenate([np.logspace(-4, np.log10(300), 3000), np.linspace(1.9, 2.1, 101),
                        64.0 / np.arange(1, 33)])
    h0, h1 = qbx.qbx_debug_hankel01(dev(z.astype(complex)))
    r0, r1 = sp.hankel1(0, z), sp.hankel1(1, z)
    tol = 5e-15 * np.maximum(1.0, z / 8)
    assert np.all(np.abs(h0.cpu().numpy() - r0) <= tol * np.abs(r0))
    assert np.all(np.abs(h1.cpu().numpy() - r1) <= tol * np.abs(r1))


def test_device_hankel_complex(cuda):
    z = np.concatenate([np.linspace(0.01, 40, 400) + 0.5j, np.linspace(0.2, 25, 100) + 1.5j,
                        np.array([1e-3 + 1e-3j, 5.99 + 0.1j, 6.01 + 0.1j, 19.99 + 0.2j, 20.01 + 0.2j])])
    h0, h1 = qbx.qbx_debug_hankel01(dev(z))
    r0, r1 = sp.hankel1(0, z), sp.hankel1(1, z)
    tol = 2e-14 * np.exp(2 * z.imag) * np.maximum(1.0, np.abs(z) / 8)
    assert np.all(np.abs(h0.cpu().numpy() - r0) <= tol * np.abs(r0))
    assert np.all(np.abs(h1.cpu().numpy() - r1) <= tol * np.abs(r1))


@pytest.mark.parametrize("k", [20 + 1j, 5 + 0.5j, 8 + 2j, 40 + 0.05j, 3 + 0.1j])
def test_device_hankel_complex_ray(cuda, k):
    """Complex k: H0, H1 at z = k rho through the amplitude table fitted for
    this k's ray (|z| >= 2; the series below), rho from 1e-3 to 3, against
    scipy.  The table's node values have the accuracy of the direct
    complex evaluation (which loses ~e^{2 Im z} to cancellation for
    |z| <= 20); above |z| = 20 they come from the asymptotic amplitude."""
    plan = qbx.Plan(16, 64, workspace_bytes=1 << 12)
    rho = np.concatenate([np.logspace(-3, np.log10(3.0), 3000), 2.0 / abs(k) * np.array([0.999, 1.0, 1.001])])
    h0, h1 = qbx.qbx_debug_hankel01_ray(plan, k, dev(rho))
    z = k * rho
    r0, r1 = sp.hankel1(0, z), sp.hankel1(1, z)
    imz = np.minimum(z.imag, 20.0 * np.sin(np.angle(k)))
    tol = 6e-14 * np.exp(2 * imz) * np.maximum(1.0, np.abs(z) / 8)
    e0 = np.abs(h0.cpu().numpy() - r0) / np.abs(r0)
    e1 = np.abs(h1.cpu().numpy() - r1) / np.abs(r1)
    assert np.all(e0 <= tol), (e0 / tol).max()
    assert np.all(e1 <= tol), (e1 / tol).max()
    # a second k on the same plan remakes the table
    k2 = k.real + 2j * k.imag
    g0, _ = qbx.qbx_debug_hankel01_ray(plan, k2, dev(rho))
    r2 = sp.hankel1(0, k2 * rho)
    imz2 = np.minimum((k2 * rho).imag, 20.0 * np.sin(np.angle(k2)))
    assert np.all(np.abs(g0.cpu().numpy() - r2) / np.abs(r2)
                  <= 6e-14 * np.exp(2 * imz2) * np.maximum(1.0, np.abs(k2 * rho) / 8))


def test_device_besselj(cuda):
    z = np.concatenate([np.linspace(1e-4, 12, 500), np.linspace(0.05, 6, 60) + 0.4j])
    nmax = 20
    J = qbx.qbx_debug_besselj(dev(z), nmax).cpu().numpy()
    for n in range(nmax + 1):
        ref = sp.jv(n, z)
        assert np.all(np.abs(J[:, n] - ref) <= 4e-15 * np.exp(np.abs(z.imag))), n


# ---------------------------------------------------------------------------
# a0, a1: geometry and oversampling
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("curve,M", [(W.starfish(), 37), (W.ellipse(3.0), 50), (W.circle(1.7), 5)])
def test_geometry_matches_oracle(cuda, curve, M):
    plan, g, go = make(curve, M)
    for name in ("src_x", "src_y", "src_nx", "src_ny", "src_w", "tgt_x", "tgt_y", "tgt_nx", "tgt_ny",
                 "tgt_w", "panel_h", "ctr_x", "ctr_y", "ctr_r", "ctr_ratio"):
        assert rel(g[name], go[name]) < 1e-14, name


def test_upsample_matches_oracle(cuda):
    plan, g, go = make(W.starfish(), 19, nrhs=3)
    d = W.complex_gaussian(11, g.n_tgt * 3).reshape(g.n_tgt, 3)
    got = qbx.qbx_upsample(plan, g, dev(d))
    assert rel(got, oracle.upsample(go, d)) < 1e-13


# ---------------------------------------------------------------------------
# a4 (unfused) and a5 + a6
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", [qbx.OP_S, qbx.OP_D])
@pytest.mark.parametrize("k", [5.0, 5 + 0.5j])
def test_form_locals_matches_oracle(cuda, kind, k):
    p, nrhs = 9, 2
    plan, g, go = make(W.starfish(), 10, nrhs=nrhs, p=p)
    wd = W.complex_gaussian(21, g.n_src * nrhs).reshape(g.n_src, nrhs)
    got = qbx.qbx_form_locals(plan, g, kind, qbx.SIDE_TWO, k, p, dev(wd))
    ref = oracle.form_locals(go, kind, oracle.SIDE_TWO, k, p, wd)
    # per order l: orders differ in magnitude by many decades
    for l in range(2 * p + 1):
        assert rel(got[:, l, :], ref[:, l, :]) < TOL, l


@pytest.mark.parametrize("what", [qbx.VALUE, qbx.GRAD])
@pytest.mark.parametrize("k", [20.0, 3 + 0.7j])
def test_eval_locals_matches_oracle(cuda, what, k):
    p, nrhs = 12, 2
    plan, g, go = make(W.starfish(), 11, nrhs=nrhs, p=p)
    nc = 2 * g.n_tgt
    alpha = W.complex_gaussian(31, nc * (2 * p + 1) * nrhs).reshape(nc, 2 * p + 1, nrhs)
    got = qbx.qbx_eval_locals(plan, g, qbx.SIDE_TWO, k, p, dev(alpha), what)
    ref = oracle.eval_locals(go, oracle.SIDE_TWO, k, p, alpha, what)
    assert rel(got, ref) < TOL
    # explicit off-surface targets inside the disks
    rng = np.random.default_rng(4)
    ectr = rng.integers(0, nc, 300).astype(np.int32)
    ang = rng.uniform(0, 2 * np.pi, 300)
    rad = rng.uniform(0, 1, 300) * go["ctr_r"][ectr]
    ex = go["ctr_x"][ectr] + rad * np.cos(ang)
    ey = go["ctr_y"][ectr] + rad * np.sin(ang)
    got = qbx.qbx_eval_locals(plan, g, qbx.SIDE_TWO, k, p, dev(alpha), what, dev(ex), dev(ey), dev(ectr))
    ref = oracle.eval_locals(go, oracle.SIDE_TWO, k, p, alpha, what, ex, ey, ectr)
    assert rel(got, ref) < TOL


# ---------------------------------------------------------------------------
# the fused apply (a1-a7)
# ---------------------------------------------------------------------------
def test_apply_starfish_32_panels(cuda):
    """Starfish 1 + 0.25 cos 5t, 32 panels x 16 nodes, 4x sources, k = 5, p = 8,
    interior centres, sigma = cos 3t + 0.5 i sin t: S and D (one-sided and PV)."""
    wl = W.cfg1()
    plan, g, go = make(wl.curve, wl.M, p=wl.p)
    dens = wl.dens(g.t_tgt)
    for op in (qbx.OP_S, qbx.OP_D, qbx.OP_GRAD_S):
        for limit in (qbx.LIMIT_ONE_SIDED, qbx.LIMIT_PV):
            got = qbx.qbx_apply(plan, g, op, qbx.SIDE_INT, limit, wl.k, wl.p, dev(dens))
            ref = oracle.apply(go, op, oracle.SIDE_INT, limit, wl.k, wl.p, dens)
            assert rel(got, ref) < TOL, (op, limit)
    qbx.qbx_sync_status(plan)


@pytest.mark.parametrize("op", [qbx.OP_S, qbx.OP_D, qbx.OP_GRAD_S])
@pytest.mark.parametrize("side,limit", [(qbx.SIDE_INT, qbx.LIMIT_ONE_SIDED), (qbx.SIDE_EXT, qbx.LIMIT_PV),
                                        (qbx.SIDE_TWO, qbx.LIMIT_ONE_SIDED)])
@pytest.mark.parametrize("k,p,nrhs", [(7.0, 10, 1), (4 + 0.6j, 6, 3), (11.0, 0, 2)])
def test_apply_variants_ragged(cuda, op, side, limit, k, p, nrhs):
    """13 panels: 208 targets (416 centres = 3 tiles + 32), 832 sources (6.5 tiles)."""
    plan, g, go = make(W.starfish(0.2, 3), 13, nrhs=nrhs, p=p)
    dens = W.complex_gaussian(7, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    got = qbx.qbx_apply(plan, g, op, side, limit, k, p, dev(dens))
    ref = oracle.apply(go, op, side, limit, k, p, dens)
    assert rel(got, ref) < TOL


ALL_SUBSETS = [(0, 1), (0, 2), (1, 2), (0, 1, 2), (0,), (1,), (2,)]


@pytest.mark.parametrize("ops", ALL_SUBSETS)
@pytest.mark.parametrize("side,limit,k,nrhs", [(qbx.SIDE_TWO, 0, 8.0, 1), (qbx.SIDE_INT, 1, 3 + 0.4j, 6),
                                               (qbx.SIDE_EXT, 1, 12.0, 3)])
def test_apply_ops_subsets(cuda, ops, side, limit, k, nrhs):
    """One pass for several operators, each with its own density, 11 panels
    (176 targets; 352 centres two-sided), 704 sources; 6 rhs = 2 launches."""
    p = 9
    plan, g, go = make(W.starfish(0.3, 4), 11, nrhs=nrhs, p=p, extra_ctr=2)
    dens = {o: W.complex_gaussian(40 + o, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs) for o in ops}
    got = qbx.qbx_apply_ops(plan, g, ops, side, limit, k, p, {o: dev(dens[o]) for o in ops})
    for o in ops:
        ref = oracle.apply(go, o, side, limit, k, p, dens[o])
        assert rel(got[o], ref) < TOL, o


@pytest.mark.parametrize("ops", ALL_SUBSETS)
@pytest.mark.parametrize("side,limit,k", [(qbx.SIDE_TWO, 0, 8.0), (qbx.SIDE_INT, 1, 3 + 0.4j),
                                          (qbx.SIDE_EXT, 0, 12.0)])
def test_apply_ops_one_density(cuda, ops, side, limit, k):
    """One rhs of one density for every operator takes the weighted-seed
    instance (the density multiplies H0, H1); the same values in separate
    arrays take the per-pair instance.  Both against the oracle, and against
    each other to rounding: 11 panels, ragged centre and source tiles."""
    p = 9
    plan, g, go = make(W.starfish(0.3, 4), 11, nrhs=1, p=p, extra_ctr=2)
    dens = W.complex_gaussian(77, g.n_tgt).reshape(g.n_tgt, 1)
    d = dev(dens)
    one = qbx.qbx_apply_ops(plan, g, ops, side, limit, k, p, d)
    sep = qbx.qbx_apply_ops(plan, g, ops, side, limit, k, p, {o: d.clone() for o in ops})
    qbx.qbx_sync_status(plan)
    for o in ops:
        ref = oracle.apply(go, o, side, limit, k, p, dens)
        assert rel(one[o], ref) < TOL, o
        assert rel(sep[o], ref) < TOL, o
        assert rel(one[o], sep[o].cpu().numpy()) < 1e-13, o


def test_apply_many_rhs(cuda):
    nrhs = 11
    plan, g, go = make(W.ellipse(2.0), 9, nrhs=nrhs)
    dens = W.complex_gaussian(8, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    for op in (qbx.OP_S, qbx.OP_GRAD_S):
        got = qbx.qbx_apply(plan, g, op, qbx.SIDE_TWO, 0, 6.0, 9, dev(dens))
        ref = oracle.apply(go, op, oracle.SIDE_TWO, 0, 6.0, 9, dens)
        assert rel(got, ref) < TOL


def test_apply_full_size_every_target(cuda):
    """Starfish, 256 panels (4096 targets, 16384 sources), k = 20, p = 12, both
    sides (8192 centres), S, D and grad S, CN(0,1) density (seed 2): the launch
    configuration of the benchmark (one pass for all operators), and each
    operator alone, against the oracle at every target."""
    wl = W.cfg2()
    plan, g, go = make(wl.curve, wl.M, p=wl.p)
    dens = wl.dens(g.t_tgt)
    ops = (qbx.OP_S, qbx.OP_D, qbx.OP_GRAD_S)
    together = qbx.qbx_apply_ops(plan, g, ops, qbx.SIDE_TWO, 0, wl.k, wl.p, dev(dens))  # benchmark call
    assert g["ctr_ratio"].min().item() > 1.0   # every centre admissible on both sides
    for op in ops:
        ref = oracle.apply(go, op, oracle.SIDE_TWO, 0, wl.k, wl.p, dens)
        alone = qbx.qbx_apply(plan, g, op, qbx.SIDE_TWO, 0, wl.k, wl.p, dev(dens))
        for got in (together[op], alone):
            assert rel(got, ref) < TOL, op
        # the one-pass and per-operator kernels agree everywhere to rounding
        assert rel(together[op], alone.cpu().numpy()) < 1e-13
    qbx.qbx_sync_status(plan)


def test_apply_full_size_complex_k(cuda):
    """The benchmark's workload at the complex wavenumber k = 20 + 1i (S, D and
    grad S in one pass, both sides): every target against the per-operator
    kernels, and 256 seeded targets (both ends included) against the oracle
    on both sides."""
    wl = W.cfg2()
    k = 20.0 + 1.0j
    plan, g, go = make(wl.curve, wl.M, p=wl.p)
    dens = wl.dens(g.t_tgt)
    ops = (qbx.OP_S, qbx.OP_D, qbx.OP_GRAD_S)
    together = qbx.qbx_apply_ops(plan, g, ops, qbx.SIDE_TWO, 0, k, wl.p, dev(dens))
    rng = np.random.default_rng(21)
    sel = np.unique(np.concatenate([[0, g.n_tgt - 1], rng.choice(g.n_tgt, 254, replace=False)]))
    for op in ops:
        ref = oracle.apply(go, op, oracle.SIDE_TWO, 0, k, wl.p, dens, sel=sel)
        assert rel(together[op].cpu().numpy()[sel], ref) < TOL, op
        alone = qbx.qbx_apply(plan, g, op, qbx.SIDE_TWO, 0, k, wl.p, dev(dens))
        # (complex J_l and recurrences: the two kernels' rounding differs more than at real k)
        assert rel(together[op], alone.cpu().numpy()) < 1e-12
    qbx.qbx_sync_status(plan)


# ---------------------------------------------------------------------------
# a8 far targets, centre assignment
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("k", [9.0, 2 + 0.4j])
def test_far_matches_oracle(cuda, k):
    nrhs = 2
    plan, g, go = make(W.starfish(), 16, nrhs=nrhs)
    th = np.linspace(0, 2 * np.pi, 257)[:-1]
    xy = np.concatenate([np.stack([2.5 * np.cos(th), 2.5 * np.sin(th)], 1),
                         np.stack([0.3 * np.cos(th[:70]), 0.3 * np.sin(th[:70])], 1)])
    dens = W.complex_gaussian(9, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    wd = oracle.upsample(go, dens)
    wdg = qbx.qbx_upsample(plan, g, dev(dens))
    for op in (qbx.OP_S, qbx.OP_D, qbx.OP_GRAD_S):
        got = qbx.qbx_far(plan, g, op, k, wdg, dev(xy))
        ref = oracle.far(go, op, k, wd, xy)
        assert rel(got, ref) < TOL, op
        on, far = qbx.qbx_apply(plan, g, op, qbx.SIDE_INT, 0, k, 8, dev(dens), x_far=dev(xy))
        assert rel(far, ref) < TOL, op


def test_assign_centres_bit_exact(cuda):
    plan, g, go = make(W.starfish(), 12)
    rng = np.random.default_rng(2)
    xy = rng.uniform(-1.4, 1.4, size=(2000, 2))
    for side in (qbx.SIDE_INT, qbx.SIDE_EXT, qbx.SIDE_TWO):
        got = qbx.qbx_assign_centres(plan, g, side, dev(xy)).cpu().numpy()
        ref = oracle.assign_centres(go, side, xy)
        c0 = g.n_tgt if side == qbx.SIDE_EXT else 0
        ref = np.where(ref >= 0, ref - c0, -1)
        assert np.array_equal(got, ref)


# ---------------------------------------------------------------------------
# determinism, streams, edge cases and errors
# ---------------------------------------------------------------------------
def test_deterministic_and_stream_ordered(cuda):
    wl = W.cfg1()
    plan, g, go = make(wl.curve, wl.M, p=wl.p)
    d = dev(wl.dens(g.t_tgt))
    a = qbx.qbx_apply(plan, g, qbx.OP_D, qbx.SIDE_TWO, 0, wl.k, wl.p, d)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = qbx.qbx_apply(plan, g, qbx.OP_D, qbx.SIDE_TWO, 0, wl.k, wl.p, d)
    s.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("k", [14.0, 6 + 0.8j])
def test_source_split_count_leaves_the_result(cuda, k):
    """The source splits (more waves of CTAs, each over fewer sources) change
    only the order of the sums: one density, S + D + grad S in one pass, the
    same values for 1, 8, 16 and 64 requested waves (the one-density apply
    takes at least 4, 8 at complex k) and against the oracle."""
    p = 10
    plan, g, go = make(W.starfish(), 48, p=p)
    dens = W.complex_gaussian(5, g.n_tgt).reshape(g.n_tgt, 1)
    ops = (qbx.OP_S, qbx.OP_D, qbx.OP_GRAD_S)
    outs = []
    for waves in (1, 8, 16, 64):
        qbx.qbx_plan_set_min_waves(plan, waves)
        outs.append(qbx.qbx_apply_ops(plan, g, ops, qbx.SIDE_TWO, 0, k, p, dev(dens)))
    qbx.qbx_sync_status(plan)
    for bad in (0, 65):
        with pytest.raises(qbx.QBXError):
            qbx.qbx_plan_set_min_waves(plan, bad)
    for op in ops:
        ref = oracle.apply(go, op, oracle.SIDE_TWO, 0, k, p, dens)
        for out in outs:
            assert rel(out[op], ref) < TOL, op
            assert rel(out[op], outs[0][op].cpu().numpy()) < 1e-13, op


def test_single_panel_and_order_zero(cuda):
    plan, g, go = make(W.circle(1.0), 1, q_tgt=16, q_src=64)
    dens = W.density_cfg1(g.t_tgt)
    for p in (0, 1, 3):
        got = qbx.qbx_apply(plan, g, qbx.OP_S, qbx.SIDE_INT, 0, 1.5, p, dev(dens))
        ref = oracle.apply(go, oracle.OP_S, oracle.SIDE_INT, 0, 1.5, p, dens)
        assert rel(got, ref) < TOL


@pytest.mark.parametrize("k", [3.0, 2 + 0.4j])
@pytest.mark.parametrize("nrhs", [1, 3, 17])
def test_all_operators_low_orders(cuda, k, nrhs):
    """S, D and grad S in one pass at the orders where D's sum by parts
    reduces to its end terms (p = 0, 1, 2): one density with weighted seeds
    (1 rhs), per-pair kernel values (3 rhs) and the group kernel (17 rhs),
    both sides, against the oracle."""
    plan, g, go = make(W.ellipse(2.0), 9, nrhs=nrhs)   # every centre admissible
    dens = W.complex_gaussian(40 + nrhs, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    ops = (qbx.OP_S, qbx.OP_D, qbx.OP_GRAD_S)
    for p in (0, 1, 2):
        got = qbx.qbx_apply_ops(plan, g, ops, qbx.SIDE_TWO, 0, k, p, dev(dens))
        for op in ops:
            ref = oracle.apply(go, op, oracle.SIDE_TWO, 0, k, p, dens)
            assert rel(got[op], ref) < TOL, (p, op)


def test_other_grid_sizes(cuda):
    plan, g, go = make(W.starfish(), 7, q_tgt=10, q_src=30)
    dens = W.density_cfg1(g.t_tgt)
    got = qbx.qbx_apply(plan, g, qbx.OP_D, qbx.SIDE_TWO, 0, 4.0, 7, dev(dens))
    ref = oracle.apply(go, oracle.OP_D, oracle.SIDE_TWO, 0, 4.0, 7, dens)
    assert rel(got, ref) < TOL


def test_errors_are_reported(cuda):
    plan, g, go = make(W.starfish(), 4)
    d = dev(W.density_cfg1(g.t_tgt))
    with pytest.raises(qbx.QBXError) as e:
        qbx.qbx_apply(plan, g, qbx.OP_S, qbx.SIDE_INT, 0, 5 - 1j, 4, d)
    assert e.value.code == 1
    with pytest.raises(qbx.QBXError) as e:
        qbx.qbx_apply(plan, g, qbx.OP_S, qbx.SIDE_INT, 0, 5.0, qbx.MAX_P + 1, d)
    assert e.value.code == 1
    with pytest.raises(qbx.QBXError) as e:
        qbx.qbx_apply(plan, g, qbx.OP_S, 7, 0, 5.0, 4, d)
    assert e.value.code == 1
    small = qbx.Plan(16, 64, workspace_bytes=1024)
    with pytest.raises(qbx.QBXError) as e:
        qbx.qbx_apply(small, g, qbx.OP_S, qbx.SIDE_INT, 0, 5.0, 4, d)
    assert e.value.code == 7
    bad = d.clone()
    bad[3] = complex(float("nan"), 0.0)
    qbx.qbx_apply(plan, g, qbx.OP_S, qbx.SIDE_INT, 0, 5.0, 4, bad)
    with pytest.raises(qbx.QBXError) as e:
        qbx.qbx_sync_status(plan)
    assert e.value.code == 4
    qbx.qbx_sync_status(plan)   # cleared


def test_kernel_timing_events(cuda):
    """With timing on, the plan records events around the pair-sum launch of
    every apply: the kernel time is positive, below the whole call's time,
    and the results are unchanged; with timing off the query is refused."""
    wl = W.cfg1()
    plan, g, go = make(wl.curve, wl.M, p=wl.p)
    d = dev(wl.dens(g.t_tgt))
    with pytest.raises(qbx.QBXError) as e:
        qbx.qbx_plan_kernel_ms(plan)
    assert e.value.code == 1
    ref = qbx.qbx_apply(plan, g, qbx.OP_S, qbx.SIDE_TWO, 0, wl.k, wl.p, d)
    qbx.qbx_plan_set_timing(plan, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = qbx.qbx_apply_ops(plan, g, (qbx.OP_S, qbx.OP_D), qbx.SIDE_TWO, 0, wl.k, wl.p, d)
    e1.record()
    kms = qbx.qbx_plan_kernel_ms(plan)
    e1.synchronize()
    assert 0.0 < kms <= e0.elapsed_time(e1)
    assert torch.equal(out[qbx.OP_S], ref) or rel(out[qbx.OP_S], ref.cpu().numpy()) < 1e-13
    qbx.qbx_plan_set_timing(plan, False)


@pytest.mark.parametrize("side,limit", [(qbx.SIDE_INT, qbx.LIMIT_PV), (qbx.SIDE_EXT, qbx.LIMIT_ONE_SIDED),
                                        (qbx.SIDE_TWO, qbx.LIMIT_PV)])
@pytest.mark.parametrize("k,p,nrhs", [(7.0, 10, 1), (4 + 0.6j, 6, 3), (9.0, 8, 20)])
def test_apply_r_matches_oracle(cuda, side, limit, k, p, nrhs):
    """The tangential dipole R (Sec. 3.2, eq. riesz-def) on 13 panels (ragged
    tiles), with far targets through the same call; 20 rhs take the group
    kernel."""
    plan, g, go = make(W.starfish(0.2, 3), 13, nrhs=nrhs, p=p)
    dens = W.complex_gaussian(17, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    xy = np.array([[0.1, 0.05], [2.5, 0.3], [-1.9, -2.2], [0.0, 1.6]])
    got, far = qbx.qbx_apply(plan, g, qbx.OP_R, side, limit, k, p, dev(dens), x_far=dev(xy))
    qbx.qbx_sync_status(plan)
    assert rel(got, oracle.apply(go, oracle.OP_R, side, limit, k, p, dens)) < TOL
    assert rel(far, oracle.far(go, oracle.OP_R, k, oracle.upsample(go, dens), xy)) < TOL
    wd = qbx.qbx_upsample(plan, g, dev(dens))
    assert rel(qbx.qbx_far(plan, g, qbx.OP_R, k, wd, dev(xy)), far.cpu().numpy()) < 1e-13


@pytest.mark.parametrize("q_src", [16, 64])
def test_sqrt_h_radius_rule(cuda, q_src):
    """r = c sqrt(h) (qbx_geometry_rule): centres and radii as the oracle's,
    and S, D, grad S on them, with and without source oversampling."""
    cur, M, k, p, c = W.starfish(0.2, 3), 20, 6.0, 10, 0.3
    plan = qbx.Plan(16, q_src, n_src=M * q_src, n_ctr=2 * M * 16, ncoef=4, nrhs=2)
    g = qbx.qbx_geometry(plan, cur, cur.edges(M), c, qbx.RADIUS_SQRT_H)
    go = oracle.geometry(cur, cur.edges(M), 16, q_src, c, oracle.RADIUS_SQRT_H)
    for name in ("ctr_x", "ctr_y", "ctr_r"):
        assert rel(g[name], go[name]) < 1e-14, name
    dens = W.complex_gaussian(21, g.n_tgt * 2).reshape(g.n_tgt, 2)
    got = qbx.qbx_apply_ops(plan, g, (0, 1, 2), qbx.SIDE_TWO, 0, k, p, dev(dens))
    for o in (0, 1, 2):
        assert rel(got[o], oracle.apply(go, o, qbx.SIDE_TWO, 0, k, p, dens)) < TOL, o
    with pytest.raises(qbx.QBXError):
        qbx.qbx_geometry(plan, cur, cur.edges(M), c, 7)


@pytest.mark.parametrize("side,limit", [(qbx.SIDE_INT, qbx.LIMIT_PV), (qbx.SIDE_EXT, qbx.LIMIT_PV),
                                        (qbx.SIDE_EXT, qbx.LIMIT_ONE_SIDED), (qbx.SIDE_TWO, qbx.LIMIT_PV)])
@pytest.mark.parametrize("k,p,nrhs", [(7.0, 10, 1), (4 + 0.6j, 6, 3), (5.0, 1, 2), (6.0, 0, 1), (8.0, 9, 5)])
def test_apply_grad_d_matches_oracle(cuda, side, limit, k, p, nrhs):
    """grad D (Sec. 3.2, eq. dlpderiv) on 13 panels, the tangential jump for
    the PV: storage-free sums for 1-3 rhs and p >= 1 (p = 1: no interior
    orders, only the edge orders), stored coefficients and the expansion's
    gradient otherwise (p = 0, 5 rhs)."""
    plan, g, go = make(W.starfish(0.2, 3), 13, nrhs=nrhs, p=p)
    dens = W.complex_gaussian(19, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    got = qbx.qbx_apply(plan, g, qbx.OP_GRAD_D, side, limit, k, p, dev(dens))
    qbx.qbx_sync_status(plan)
    assert got.shape == (g.n_tgt, 2, nrhs)
    assert rel(got, oracle.apply(go, oracle.OP_GRAD_D, side, limit, k, p, dens)) < TOL


@pytest.mark.parametrize("k,p", [(7.0, 10), (3 + 0.5j, 8), (9.0, 2)])
def test_grad_d_fused_matches_stored_coefficients(cuda, k, p):
    """The storage-free grad D (one rhs) and the stored-coefficient path (the
    same density in 4 columns) agree to rounding on every target, both
    sides."""
    plan, g, go = make(W.starfish(0.2, 3), 17, nrhs=4, p=p)
    dens = W.complex_gaussian(37, g.n_tgt).reshape(g.n_tgt, 1)
    one = qbx.qbx_apply(plan, g, qbx.OP_GRAD_D, qbx.SIDE_TWO, qbx.LIMIT_PV, k, p, dev(dens))
    four = qbx.qbx_apply(plan, g, qbx.OP_GRAD_D, qbx.SIDE_TWO, qbx.LIMIT_PV, k, p, dev(np.repeat(dens, 4, axis=1)))
    qbx.qbx_sync_status(plan)
    assert rel(one[:, :, 0], four[:, :, 0].cpu().numpy()) < 1e-12
    assert rel(one[:, :, 0], four[:, :, 3].cpu().numpy()) < 1e-12


@pytest.mark.parametrize("ops,side,limit,k,eta,nrhs", [((0, 1, 2), qbx.SIDE_TWO, 0, 7.0, 3.0, 2),
                                                       ((0,), qbx.SIDE_INT, 1, 3 + 0.5j, 5.0, 2),
                                                       ((1, 2), qbx.SIDE_EXT, 1, 9.0, 8.0, 2),
                                                       ((0, 1, 2), qbx.SIDE_TWO, 1, 7.0, 3.0, 17),
                                                       ((0, 1), qbx.SIDE_INT, 0, 3 + 0.5j, 4.0, 16)])
def test_apply_local_matches_oracle(cuda, ops, side, limit, k, eta, nrhs):
    """Near-only QBX (qbx_apply_local): the oracle's near/far split with the
    same eta; pairs exactly at the boundary may fall on either side, which
    costs at most eta^-(p+1) of a pair's kernel.  16 and 17 rhs of one
    density take the group kernel."""
    p = 10
    plan, g, go = make(W.starfish(0.2, 3), 24, nrhs=nrhs, p=p)
    dens = W.complex_gaussian(23, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    got = qbx.qbx_apply_ops(plan, g, ops, side, limit, k, p, dev(dens), eta=eta)
    qbx.qbx_sync_status(plan)
    glob = qbx.qbx_apply_ops(plan, g, ops, side, limit, k, p, dev(dens))
    for o in ops:
        assert rel(got[o], oracle.apply_local(go, o, side, limit, k, p, eta, dens)) < TOL, o
        # and it is not the global apply (every case has distant sources)
        assert rel(got[o], glob[o].cpu().numpy()) > 1e-14, o
    with pytest.raises(qbx.QBXError):
        qbx.qbx_apply_ops(plan, g, ops, side, limit, k, p, dev(dens), eta=-1.0)


@pytest.mark.parametrize("ops", [(0, 1, 2), (0,), (1, 2), (0, 1)])
@pytest.mark.parametrize("side,limit,k,eta", [(qbx.SIDE_TWO, 0, 7.0, 3.0), (qbx.SIDE_INT, 1, 3 + 0.5j, 5.0)])
def test_apply_local_one_density(cuda, ops, side, limit, k, eta):
    """Near-only QBX with one rhs of one density (weighted seeds for the
    expansion pairs and the direct pairs) against the oracle and against the
    same values in separate arrays (per-pair kernel values)."""
    p = 10
    plan, g, go = make(W.starfish(0.2, 3), 24, nrhs=1, p=p, extra_ctr=2)
    dens = W.complex_gaussian(29, g.n_tgt).reshape(g.n_tgt, 1)
    d = dev(dens)
    one = qbx.qbx_apply_ops(plan, g, ops, side, limit, k, p, d, eta=eta)
    sep = qbx.qbx_apply_ops(plan, g, ops, side, limit, k, p, {o: d.clone() for o in ops}, eta=eta)
    qbx.qbx_sync_status(plan)
    for o in ops:
        assert rel(one[o], oracle.apply_local(go, o, side, limit, k, p, eta, dens)) < TOL, o
        assert rel(one[o], sep[o].cpu().numpy()) < 1e-13, o


@pytest.mark.parametrize("k,p,nrhs", [(6.0, 40, 1), (6.0, 40, 20), (3 + 0.4j, 30, 2)])
def test_maximum_orders(cuda, k, p, nrhs):
    """The largest orders: p = QBX_MAX_P = 40 (real k; fused kernel and, with
    20 rhs, the group kernel) and p = 30 for complex k (the fused kernel's
    coefficient columns of complex J_l fill most of the shared memory), on the
    32-panel starfish, all three operators in one call."""
    assert qbx.MAX_P == 40
    cur = W.starfish()
    plan, g, go = make(cur, 32, nrhs=nrhs, p=p)
    dens = W.complex_gaussian(31, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    got = qbx.qbx_apply_ops(plan, g, (0, 1, 2), qbx.SIDE_INT, qbx.LIMIT_PV, k, p, dev(dens))
    qbx.qbx_sync_status(plan)
    for o in (0, 1, 2):
        assert rel(got[o], oracle.apply(go, o, qbx.SIDE_INT, qbx.LIMIT_PV, k, p, dens)) < TOL, o
    with pytest.raises(qbx.QBXError):
        qbx.qbx_apply_ops(plan, g, (0, 1, 2), qbx.SIDE_INT, qbx.LIMIT_PV, k, 41, dev(dens))


def _random_cases(n, seed=20240607):
    rng = np.random.default_rng(seed)
    subsets = [(0,), (1,), (2,), (0, 1), (0, 2), (1, 2), (0, 1, 2)]
    cases = []
    for _ in range(n):
        ops = subsets[rng.integers(len(subsets))]
        side = int(rng.integers(3))
        limit = int(rng.integers(2))
        kr = float(rng.uniform(1.0, 15.0))
        k = complex(kr, float(rng.uniform(0.05, 1.5))) if rng.random() < 0.5 else kr
        p = int(rng.integers(1, 13))
        nrhs = int(rng.choice([1, 1, 2, 5, 17]))
        eta = float(rng.uniform(2.5, 8.0)) if rng.random() < 0.3 else None
        M = int(rng.integers(10, 19))
        cases.append((ops, side, limit, k, p, nrhs, eta, M))
    return cases


@pytest.mark.parametrize("case", _random_cases(40))
def test_random_combinations(cuda, case):
    """Seeded random combinations of operator subset, side, limit, real or
    complex k, order, rhs count (1: weighted seeds; 17: group kernel),
    near-only eta and panel count against the oracle: the paths exercised
    together (complex-k tables with near-only, the group kernel, one
    density for several operators)."""
    ops, side, limit, k, p, nrhs, eta, M = case
    sides = (qbx.SIDE_INT, qbx.SIDE_EXT, qbx.SIDE_TWO)
    side = sides[side]
    plan, g, go = make(W.starfish(0.2, 3), M, nrhs=nrhs, p=p)
    dens = W.complex_gaussian(M + p, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    got = qbx.qbx_apply_ops(plan, g, ops, side, limit, k, p, dev(dens), eta=eta)
    qbx.qbx_sync_status(plan)
    for o in ops:
        ref = (oracle.apply_local(go, o, side, limit, k, p, eta, dens) if eta is not None
               else oracle.apply(go, o, side, limit, k, p, dens))
        assert rel(got[o], ref) < TOL, (case, o)


@pytest.mark.parametrize("seed", range(12))
def test_random_r_and_grad_d(cuda, seed):
    """Seeded random cases of R and grad D (qbx_apply): side, limit, real or
    complex k, order, rhs count (1-3: storage-free grad D; 4-5: stored
    coefficients), panel count, against the oracle."""
    rng = np.random.default_rng(1000 + seed)
    op = (qbx.OP_R, qbx.OP_GRAD_D)[seed % 2]
    side = (qbx.SIDE_INT, qbx.SIDE_EXT, qbx.SIDE_TWO)[int(rng.integers(3))]
    limit = int(rng.integers(2))
    kr = float(rng.uniform(1.0, 12.0))
    k = complex(kr, float(rng.uniform(0.05, 1.0))) if rng.random() < 0.5 else kr
    p = int(rng.integers(1, 12))
    nrhs = int(rng.integers(1, 6))
    M = int(rng.integers(10, 17))
    plan, g, go = make(W.starfish(0.2, 3), M, nrhs=nrhs, p=p)
    dens = W.complex_gaussian(seed + 7, g.n_tgt * nrhs).reshape(g.n_tgt, nrhs)
    got = qbx.qbx_apply(plan, g, op, side, limit, k, p, dev(dens))
    qbx.qbx_sync_status(plan)
    oop = oracle.OP_R if op == qbx.OP_R else oracle.OP_GRAD_D
    assert rel(got, oracle.apply(go, oop, side, limit, k, p, dens)) < TOL, (op, side, limit, k, p, nrhs, M)
