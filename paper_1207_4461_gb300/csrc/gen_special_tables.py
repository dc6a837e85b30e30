"""Generate special_tables.h: coefficient tables for the device Hankel H0, H1.

Run from this directory:  python gen_special_tables.py   (needs mpmath).
The output header is committed; the build does not run this script.

Real argument z > 0 is split in two regions.

Large z (z >= Z_SPLIT): the modulated amplitudes B_n(s) = H_n(z) e^{-i(z - pi/4)},
s = z^{-1/2}, n = 0, 1.  By Hankel's expansion (DLMF 10.17.3-10.17.5)
B_n(s) = sqrt(2/pi) s e^{-i n pi/2} (P_n(s^2) + i Q_n(s^2)) with P, Q smooth, so
B_n is smooth in s on [0, Z_SPLIT^{-1/2}] (no square root left to evaluate).
B_n is approximated piecewise on intervals of width 1/NI_PER_UNIT in s by
polynomials in u = s - s_mid.  The coefficients come from Chebyshev
interpolation of 34-digit mpmath values at the Chebyshev nodes of each
interval (converted to the monomial basis in u).  The degree is the smallest
one for which every interval is within MAX_ERR on a dense check grid.

Small z (z < Z_SPLIT): ascending series in t = (z/2)^2 (DLMF 10.2.2, 10.8.1):
  J0 = sum_m (-t)^m/(m!)^2,   J1 = (z/2) sum_m (-t)^m/(m!(m+1)!)
  Y0 = (2/pi) ln(z/2) J0 - (2/pi) sum_m psi(m+1) (-t)^m/(m!)^2
  Y1 = -2/(pi z) + (2/pi) ln(z/2) J1 - (z/(2 pi)) sum_m (psi(m+1)+psi(m+2)) (-t)^m/(m!(m+1)!)
The series coefficients are written out as exact rationals rounded to double.

Phase: e^{i(z - pi/4)} uses a table of e^{i(2 pi j/NT - pi/4)}, j < NT, and a
short Taylor polynomial of e^{i r}, |r| <= pi/NT, after Cody-Waite reduction
of z by 2 pi/NT (two-part split of the step, high part with 30 significant bits).
The polynomial (cos to r^4, sin to r^5) leaves r^6/720 < 8e-17 at NT = 512.
"""
import mpmath as mp
import numpy as np

mp.mp.dps = 40

Z_SPLIT = 2.0          # series below, amplitude fits above
NI_PER_UNIT = 256      # intervals per unit of s (a power of two)
NI = int(mp.ceil(NI_PER_UNIT / mp.sqrt(Z_SPLIT)))   # intervals covering s in [0, Z_SPLIT^-1/2]
MAX_ERR = 3.5e-16      # absolute; |B_n| <= 0.6 on the range
NT = 512               # phase table size (8 KB: with the amplitude table it stays in L1)
NSER = 14              # series terms (t <= 1: 1/(13!)^2 ~ 2.6e-20)


def amp(n, s):
    if s == 0:
        return mp.mpc(0, 0)
    z = 1 / mp.mpf(s) ** 2
    return mp.hankel1(n, z) * mp.expj(-(z - mp.pi / 4))


def fit_interval(n, a, b, deg):
    a, b = mp.mpf(a), mp.mpf(b)
    mid, half = (a + b) / 2, (b - a) / 2
    xs = [mp.cos(mp.pi * (j + mp.mpf(1) / 2) / (deg + 1)) for j in range(deg + 1)]
    vals = [amp(n, mid + half * x) for x in xs]
    out = []
    for part in (lambda v: v.real, lambda v: v.imag):
        # Chebyshev coefficients in mpmath precision
        c = []
        for kk in range(deg + 1):
            s = mp.fsum(part(vals[j]) * mp.cos(kk * mp.pi * (j + mp.mpf(1) / 2) / (deg + 1))
                        for j in range(deg + 1))
            c.append(s * (2 if kk else 1) / (deg + 1))
        # to monomials in x, then in u = half * x
        mono = [mp.mpf(0)] * (deg + 1)
        Tm2 = [mp.mpf(1)] + [mp.mpf(0)] * deg          # T0
        Tm1 = [mp.mpf(0), mp.mpf(1)] + [mp.mpf(0)] * (deg - 1)  # T1
        T = [Tm2, Tm1]
        for kk in range(2, deg + 1):
            nxt = [mp.mpf(0)] * (deg + 1)
            for j in range(deg):
                nxt[j + 1] += 2 * T[-1][j]
            for j in range(deg + 1):
                nxt[j] -= T[-2][j]
            T.append(nxt)
        for kk in range(deg + 1):
            for j in range(deg + 1):
                mono[j] += c[kk] * T[kk][j]
        out.append([mono[j] / half ** j for j in range(deg + 1)])
    return float(mid), out


def horner(coef, u):
    acc = 0.0
    for c in reversed(coef):
        acc = acc * u + c
    return acc


def check(n, a, b, mid, coefs):
    err = 0.0
    for w in np.linspace(a, b, 41):
        v = amp(n, w)
        u = (1.0 + w) - (1.0 + mid)   # the kernel forms u from s + 1
        err = max(err, abs(float(v.real) - horner([float(c) for c in coefs[0]], u)),
                  abs(float(v.imag) - horner([float(c) for c in coefs[1]], u)))
    return err


def build_amp_tables():
    width = 1.0 / NI_PER_UNIT
    for deg in range(4, 12):
        tabs, worst = {}, 0.0
        for n in (0, 1):
            rows = []
            for i in range(NI):
                a, b = i * width, (i + 1) * width
                mid, coefs = fit_interval(n, a, b, deg)
                worst = max(worst, check(n, a, b, mid, coefs))
                rows.append((mid, coefs))
            tabs[n] = rows
        print(f"degree {deg}: worst abs error {worst:.2e}")
        if worst <= MAX_ERR:
            return deg, width, tabs, worst
    raise RuntimeError("no degree met the error target")


def series_tables():
    def psi(m):  # digamma at positive integers
        return -mp.euler + mp.fsum(mp.mpf(1) / j for j in range(1, m))
    j0 = [(-1) ** m / mp.factorial(m) ** 2 for m in range(NSER)]
    j1 = [(-1) ** m / (mp.factorial(m) * mp.factorial(m + 1)) for m in range(NSER)]
    y0 = [-(2 / mp.pi) * psi(m + 1) * (-1) ** m / mp.factorial(m) ** 2 for m in range(NSER)]
    y1 = [-(1 / (2 * mp.pi)) * (psi(m + 1) + psi(m + 2)) * (-1) ** m /
          (mp.factorial(m) * mp.factorial(m + 1)) for m in range(NSER)]
    return j0, j1, y0, y1


def fmt(x):
    return repr(float(x))


def main():
    deg, width, tabs, worst = build_amp_tables()
    j0, j1, y0, y1 = series_tables()
    step = 2 * mp.pi / NT
    # high part of the reduction step with 30 significant bits
    e = mp.floor(mp.log(step, 2))
    hi = mp.floor(step * mp.mpf(2) ** (29 - e)) / mp.mpf(2) ** (29 - e)
    lo = step - hi
    lines = []
    lines.append("// Generated by gen_special_tables.py -- do not edit.")
    lines.append("// Device Hankel H0/H1 tables (real argument); see the generator's docstring.")
    lines.append("#pragma once")
    lines.append("// QBX_HK_GQUAL / QBX_HK_CQUAL: storage qualifiers chosen by the includer")
    lines.append("// (device global memory for lane-divergent tables, constant memory for")
    lines.append("// uniformly indexed ones).")
    lines.append("#ifndef QBX_HK_GQUAL")
    lines.append("#define QBX_HK_GQUAL static const")
    lines.append("#endif")
    lines.append("#ifndef QBX_HK_CQUAL")
    lines.append("#define QBX_HK_CQUAL static const")
    lines.append("#endif")
    lines.append(f"#define QBX_HK_ZSPLIT {fmt(Z_SPLIT)}")
    lines.append(f"#define QBX_HK_NI {NI}")
    lines.append(f"#define QBX_HK_DEG {deg}")
    lines.append(f"#define QBX_HK_S_MAX {fmt(mp.sqrt(1 / mp.mpf(Z_SPLIT)))}")
    lines.append(f"#define QBX_HK_LOG2_PER_UNIT {int(mp.log(NI_PER_UNIT, 2))}")
    lines.append(f"#define QBX_HK_NSER {NSER}")
    lines.append(f"#define QBX_HK_NT {NT}")
    lines.append(f"#define QBX_HK_RED_SCALE {fmt(NT / (2 * mp.pi))}")
    lines.append(f"#define QBX_HK_RED_HI {fmt(hi)}")
    lines.append(f"#define QBX_HK_RED_LO {fmt(lo)}")
    lines.append(f"// worst fitted amplitude error on the check grid: {worst:.2e}")
    # amplitude table: [NI][DEG+1][4 parts Re B0, Im B0, Re B1, Im B1] (the four
    # coefficients of one degree adjacent: two 16-byte loads), plus 1 + mids
    lines.append(f"QBX_HK_GQUAL double qbx_hk_mid1[{NI}] = {{")
    lines.append("  " + ", ".join(fmt(1.0 + tabs[0][i][0]) for i in range(NI)) + "};")
    lines.append(f"QBX_HK_GQUAL __align__(16) double qbx_hk_amp[{NI}][{deg + 1}][4] = {{")
    for i in range(NI):
        rows = []
        for d in range(deg + 1):
            rows.append("{" + ", ".join(fmt(tabs[n][i][1][part][d]) for n in (0, 1) for part in (0, 1)) + "}")
        lines.append("  {" + ", ".join(rows) + "},")
    lines.append("};")
    lines.append(f"QBX_HK_CQUAL double qbx_hk_ser[4][{NSER}] = {{")
    for arr in (j0, j1, y0, y1):
        lines.append("  {" + ", ".join(fmt(c) for c in arr) + "},")
    lines.append("};")
    lines.append(f"QBX_HK_GQUAL __align__(16) double qbx_hk_phase[{NT}][2] = {{")
    for j in range(NT):
        a = 2 * mp.pi * j / NT - mp.pi / 4
        lines.append(f"  {{{fmt(mp.cos(a))}, {fmt(mp.sin(a))}}},")
    lines.append("};")
    with open("special_tables.h", "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote special_tables.h, degree", deg)


if __name__ == "__main__":
    main()
