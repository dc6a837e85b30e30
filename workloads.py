"""Seeded synthetic inputs shared by the GPU path's tests/bench and the oracle.

This module holds no arithmetic of the QBX method: only curve
parametrisations (gamma(t), gamma'(t)), densities, panel edges in the curve
parameter, a counter-based random generator, and the named workloads.  Both
sides evaluate the curves at their own Gauss-Legendre nodes.

Random numbers: splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) -> uniform doubles from the top
53 bits -> Box-Muller for Gaussians.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n successive outputs of splitmix64 started at `seed` (uint64; numpy
    uint64 arithmetic wraps modulo 2^64 as the generator requires)."""
    s = np.uint64(int(seed) & _MASK) + np.arange(1, n + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    z = (s ^ (s >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int) -> np.ndarray:
    """n uniform doubles in (0, 1) (top 53 bits, offset by half an ulp)."""
    u = splitmix64(seed, n) >> np.uint64(11)
    return (u.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def complex_gaussian(seed: int, n: int) -> np.ndarray:
    """n i.i.d. CN(0,1) samples (E|z|^2 = 1), Box-Muller on splitmix64 uniforms."""
    u = uniform(seed, 2 * n)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    th = 2.0 * math.pi * u[1::2]
    return (r * np.cos(th) + 1j * r * np.sin(th)) / math.sqrt(2.0)


# ----------------------------------------------------------------------------
# Curves: callables t -> (gamma [n,2], dgamma/dt [n,2]); counter-clockwise.
# ----------------------------------------------------------------------------
@dataclass
class Curve:
    name: str
    t0: float
    t1: float
    fn: object = field(repr=False)

    def __call__(self, t):
        return self.fn(np.asarray(t, dtype=np.float64))

    def edges(self, M: int) -> np.ndarray:
        """M panels equispaced in the curve parameter."""
        return np.linspace(self.t0, self.t1, M + 1)


def _polar(rf, drf):
    def fn(t):
        r, dr = rf(t), drf(t)
        c, s = np.cos(t), np.sin(t)
        g = np.stack([r * c, r * s], axis=-1)
        dg = np.stack([dr * c - r * s, dr * s + r * c], axis=-1)
        return g, dg
    return fn


def starfish(amp: float = 0.25, arms: int = 5) -> Curve:
    """r(t) = 1 + amp cos(arms t), t in [0, 2 pi)."""
    return Curve(f"starfish(1+{amp}cos{arms}t)", 0.0, 2 * math.pi,
                 _polar(lambda t: 1.0 + amp * np.cos(arms * t),
                        lambda t: -amp * arms * np.sin(arms * t)))


def circle(R: float = 1.0) -> Curve:
    return Curve(f"circle(R={R})", 0.0, 2 * math.pi,
                 _polar(lambda t: R + 0.0 * t, lambda t: 0.0 * t))


def ellipse(alpha: float) -> Curve:
    """The paper's ellipse family gamma(t) = (cos 2 pi t, sin(2 pi t)/alpha), t in [0,1)."""
    w = 2 * math.pi

    def fn(t):
        g = np.stack([np.cos(w * t), np.sin(w * t) / alpha], axis=-1)
        dg = np.stack([-w * np.sin(w * t), w * np.cos(w * t) / alpha], axis=-1)
        return g, dg
    return Curve(f"ellipse({alpha})", 0.0, 1.0, fn)


def fourier_curve(a, b) -> Curve:
    """r(t) = 1 + sum_m (a_m cos m t + b_m sin m t), m = 1..len(a)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m = np.arange(1, a.size + 1, dtype=np.float64)

    def rf(t):
        return 1.0 + (a[None, :] * np.cos(np.outer(t, m)) + b[None, :] * np.sin(np.outer(t, m))).sum(-1)

    def drf(t):
        return (m[None, :] * (-a[None, :] * np.sin(np.outer(t, m)) + b[None, :] * np.cos(np.outer(t, m)))).sum(-1)
    return Curve("fourier", 0.0, 2 * math.pi, _polar(rf, drf))


def teardrop(right_angle: bool = False) -> Curve:
    """gamma(t) = 1.7 (sin(pi t) - 0.5, c cos(pi t)(pi t - pi) pi t), t in [0, 1],
    a closed counter-clockwise curve with one corner at t = 0 = 1.  c = 1/2 is
    the paper's teardrop (Sec. 4.2; interior angle 2 atan(pi/2), about 115
    degrees); c = 1/pi (right_angle=True) gives exactly 90 degrees, where the
    interior centres of the targets next to the corner lie on the opposite
    arm."""
    c = 1.0 / math.pi if right_angle else 0.5
    pi = math.pi

    def fn(t):
        x = 1.7 * (np.sin(pi * t) - 0.5)
        y = 1.7 * c * np.cos(pi * t) * (pi * t - pi) * pi * t
        dx = 1.7 * pi * np.cos(pi * t)
        dy = 1.7 * c * (-pi * np.sin(pi * t) * (pi * t - pi) * pi * t + np.cos(pi * t) * pi * (2 * pi * t - pi))
        return np.stack([x, y], -1), np.stack([dx, dy], -1)
    return Curve("teardrop90" if right_angle else "teardrop", 0.0, 1.0, fn)


def dyadic_edges(m_base: int, levels: int, t0: float = 0.0, t1: float = 1.0) -> np.ndarray:
    """m_base panels equispaced in t, then the panel next to each end (the
    corner at t0 = t1) bisected `levels` times toward the end: m_base +
    2 levels panels, neighbours differing in length by at most 2."""
    e = np.linspace(t0, t1, m_base + 1)
    h = e[1] - e[0]
    left = [t0 + h / 2 ** j for j in range(levels, 0, -1)]
    right = [t1 - h / 2 ** j for j in range(1, levels + 1)]
    return np.concatenate([[t0], left, e[1:-1], right, [t1]])


# ----------------------------------------------------------------------------
# Densities on the target grid, as functions of the curve parameter.
# ----------------------------------------------------------------------------
def density_cfg1(t):
    """sigma(t) = cos 3t + 0.5 i sin t."""
    t = np.asarray(t, dtype=np.float64)
    return np.cos(3 * t) + 0.5j * np.sin(t)


def fourier_mode(m: int):
    def f(t):
        return np.exp(1j * m * np.asarray(t, dtype=np.float64))
    return f


# ----------------------------------------------------------------------------
# Named workloads.  Sizes: n_tgt = M*16 targets, n_src = M*64 sources.
# ----------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    curve: Curve
    M: int
    k: complex
    p: int
    q_tgt: int = 16
    q_src: int = 64
    r_factor: float = 0.5
    sides: str = "int"          # "int", "ext" or "two"
    ops: tuple = ("S", "D")
    nrhs: int = 1
    density: str = "cfg1"       # "cfg1" or "gauss"
    seed: int = 0

    @property
    def n_tgt(self):
        return self.M * self.q_tgt

    @property
    def n_src(self):
        return self.M * self.q_src

    @property
    def n_ctr(self):
        return self.n_tgt * (2 if self.sides == "two" else 1)

    def terms_per_op(self):
        """centre x source x order(2p+1) x rhs."""
        return self.n_ctr * self.n_src * (2 * self.p + 1) * self.nrhs

    def dens(self, t_tgt):
        if self.density == "cfg1":
            d = density_cfg1(t_tgt)
            return np.repeat(d[:, None], self.nrhs, axis=1)
        g = complex_gaussian(self.seed, self.n_tgt * self.nrhs)
        return g.reshape(self.n_tgt, self.nrhs)


def cfg1() -> Workload:
    """Starfish 1 + 0.25 cos 5t, 32 panels x 16 targets, 4x sources, k=5, p=8,
    interior centres, sigma = cos 3t + 0.5 i sin t; S and D."""
    return Workload("starfish-M32-k5-p8-int", starfish(), 32, 5.0, 8, sides="int",
                    ops=("S", "D"), density="cfg1")


@dataclass
class BatchWorkload:
    """Many random smooth curves r(t) = 1 + sum_{m=1..8} (a_m cos mt + b_m sin mt),
    a_m, b_m ~ U(-0.04, 0.04), panel counts M ~ U{m_lo..m_hi}, k ~ U(k_lo, k_hi),
    nrhs CN(0,1) densities per curve, interior centres, S and D."""
    name: str
    n_inst: int
    p: int
    nrhs: int
    seed: int
    m_lo: int = 16
    m_hi: int = 512
    k_lo: float = 1.0
    k_hi: float = 40.0
    q_tgt: int = 16
    q_src: int = 64
    ops: tuple = ("S", "D")
    sides: str = "int"

    def instances(self):
        """[(curve, M, k)] drawn from splitmix64 with this workload's seed."""
        u = uniform(self.seed, self.n_inst * 18)
        out = []
        for i in range(self.n_inst):
            v = u[18 * i:18 * i + 18]
            a = -0.04 + 0.08 * v[0:8]
            b = -0.04 + 0.08 * v[8:16]
            M = self.m_lo + min(int(v[16] * (self.m_hi - self.m_lo + 1)), self.m_hi - self.m_lo)
            k = self.k_lo + (self.k_hi - self.k_lo) * v[17]
            out.append((fourier_curve(a, b), M, float(k)))
        return out

    def dens(self, i, n_tgt):
        """Curve i's densities on its target grid, [n_tgt][nrhs]."""
        return complex_gaussian(self.seed * 1000003 + 17 * i + 1, n_tgt * self.nrhs).reshape(n_tgt, self.nrhs)


def cfg3() -> BatchWorkload:
    """64 random curves, 16..512 panels x 16 nodes, k ~ U(1, 40), p = 10,
    32 CN(0,1) densities each (seed 3), interior centres, S and D."""
    return BatchWorkload("fourier-batch-64-p10-32rhs", 64, 10, 32, 3)


def cfg2() -> Workload:
    """Starfish, 256 panels (4096 targets, 16384 sources), k=20, p=12, interior
    and exterior centres (8192), S, D and grad S, CN(0,1) density, seed 2."""
    return Workload("starfish-M256-k20-p12-two", starfish(), 256, 20.0, 12, sides="two",
                    ops=("S", "D", "GRAD_S"), density="gauss", seed=2)
