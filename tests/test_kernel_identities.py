"""Identities the CUDA order loops rely on, checked on the CPU against their
definitions in 50-digit arithmetic (mpmath), at random pair geometries.

For one (centre, source) pair the double-layer Graf sum (Sec. 3.2, the
normal derivative of the addition theorem) is
    D = k a T + (2 b/rho) D2,
    T = J0 H0' + 2 sum_{l=1..p} J_l cos(l psi) H_l',   D2 = sum l J_l sin(l psi) H_l,
with J_l = J_l(k r), H_l = H_l(k rho), H_l' = (H_{l-1} - H_{l+1})/2,
H_0' = -H_1, a = n.e_rho, b = n.e_theta.  The kernels never form T from this
definition:
  * with grad S, from grad S's sum A = sum_{l>=0} G_l cos(l psi) H_l
    (G_l = J_{l-1} - J_{l+1}, G_0 = -J_1):
        T = -cos psi A - (2 sin psi/(k r)) D2 - E,
        E = J_{p+1} cos((p+1) psi) H_p + J_p cos(p psi) H_{p+1};
  * without it (the source-position gradient), by parts:
        T = t_1 H_0 + sum_{m=1..p-1} (t_{m+1} - t_{m-1}) H_m - t_{p-1} H_p - t_p H_{p+1},
    t_m = J_m cos(m psi), t_0 = J_0 (t_1 = 0 at p = 0).
Both must equal the definition for every order p, real and complex k."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")


def cases(seed, n):
    rng = np.random.default_rng(seed)
    for i in range(n):
        k = [20.0, 20 + 1j, 3.0, 40 + 0.5j][i % 4]
        p = [0, 1, 2, 7, 12, 14][i % 6]
        r = 10 ** rng.uniform(-3, -1)
        rho = r * 10 ** rng.uniform(-0.1, 2.0)
        psi = rng.uniform(-np.pi, np.pi)
        a_ang = rng.uniform(-np.pi, np.pi)
        yield k, p, r, rho, psi, np.cos(a_ang), np.sin(a_ang)


def columns(k, p, r, rho):
    kk = mp.mpc(k)
    J = [mp.besselj(l, kk * r) for l in range(p + 2)]
    H = [mp.hankel1(l, kk * rho) for l in range(p + 2)]
    return kk, J, H


def t_definition(J, H, p, psi):
    Hd = [-H[1]] + [(H[l - 1] - H[l + 1]) / 2 for l in range(1, p + 1)]
    return J[0] * Hd[0] + sum(2 * J[l] * mp.cos(l * psi) * Hd[l] for l in range(1, p + 1))


@pytest.mark.parametrize("seed", [1, 2])
def test_t_from_grad_s_sums(seed):
    mp.mp.dps = 50
    for k, p, r, rho, psi, a, b in cases(seed, 48):
        kk, J, H = columns(k, p, r, rho)
        psi = mp.mpf(psi)
        G = [-J[1]] + [J[l - 1] - J[l + 1] for l in range(1, p + 1)]
        A = sum(G[l] * mp.cos(l * psi) * H[l] for l in range(p + 1))
        D2 = sum(l * J[l] * mp.sin(l * psi) * H[l] for l in range(1, p + 1))
        E = J[p + 1] * mp.cos((p + 1) * psi) * H[p] + J[p] * mp.cos(p * psi) * H[p + 1]
        terms = [-mp.cos(psi) * A, -2 * mp.sin(psi) / (kk * r) * D2, -E]
        ref = t_definition(J, H, p, psi)
        # 50 digits, compared on the scale of the largest of the three terms
        # (they cancel to the size of T when the source is near the centre)
        scale = max(abs(x) for x in terms + [ref])
        assert abs(sum(terms) - ref) <= mp.mpf(10) ** -30 * scale, (k, p, r, rho)
        # and D as the kernels combine it
        d = kk * a * ref + 2 * b / rho * D2
        d_new = -kk * a * mp.cos(psi) * A + 2 * (b / rho - a * mp.sin(psi) / r) * D2 - kk * a * E
        assert abs(d - d_new) <= mp.mpf(10) ** -30 * max(abs(kk * a) * scale, abs(2 * D2 / rho)), (k, p)


@pytest.mark.parametrize("seed", [3])
def test_t_by_parts(seed):
    mp.mp.dps = 50
    for k, p, r, rho, psi, a, b in cases(seed, 48):
        kk, J, H = columns(k, p, r, rho)
        psi = mp.mpf(psi)
        t = [J[0]] + [J[m] * mp.cos(m * psi) for m in range(1, p + 1)] + [mp.mpf(0)]   # t_{p+1} = 0
        if p == 0:
            T = -t[0] * H[1]
        else:
            T = t[1] * H[0] + sum((t[m + 1] - t[m - 1]) * H[m] for m in range(1, p)) - t[p - 1] * H[p] - t[p] * H[p + 1]
        ref = t_definition(J, H, p, psi)
        assert abs(T - ref) <= mp.mpf(10) ** -30 * abs(ref), (k, p)
