"""Generate pw_quadrature.h: the quadratures of the plane-wave (exponential) M2L.

For two points in boxes of width w that are well separated along an axis (box centres at
least two widths apart on it), write the separation in box units as (x, y, z) with z in
[1, 4] along that axis and rho = |(x, y)| <= 4 sqrt(2) across it.  The kernels of Eq. 3
have the plane-wave representations (a Sommerfeld-type integral; for kappa = 0 it is the
Laplace one that the FMM97 exponential expansions discretise)

    exp(-k r) / r = int_0^inf exp(-(k + t) z) J0(sqrt(t^2 + 2 k t) rho) dt,     k = kappa w,
    J0(s rho)     = (1 / 2 pi) int_0^{2 pi} exp(i s (x cos a + y sin a)) da.

The t-integral is discretised by a quadrature (t_j, w_j) per band of k, the a-integral by
the trapezoid rule with M_j points (M_j even, so that the points come in opposite pairs
whose terms are complex conjugates and only M_j / 2 are kept).  The bound asked of the
whole double sum is an absolute error below EPS times 1/r for every z in [1, 4],
rho <= 4 sqrt(2) and k in the band -- the far-field sums add Laplace- and Yukawa-kernel
terms, so 1/r is the scale of each term.

The t-nodes are chosen from a fine composite Gauss-Legendre rule on [0, 60] by a
column-pivoted QR of the sampled integrand family (the numerical rank of the family at
EPS), the weights by least squares on those columns; M_j is the smallest even count whose
trapezoid error, weighted by w_j exp(-(k + t_j)), stays below 4 EPS / n (n nodes) of the
smallest 1/r -- per-node bounds that do not add up coherently, so the check at the end
evaluates the whole discrete double sum on fresh samples and must stay below EPS.

Run:  python pw_quadrature.py  (writes pw_quadrature.h next to this file; numpy + scipy)
"""
import os

import numpy as np
import scipy.linalg as la
import scipy.special as sp

EPS = 1e-6
RHO_MAX = 4.0 * np.sqrt(2.0)
Z_MIN, Z_MAX = 1.0, 4.0
BANDS = [(0.0, 0.0), (0.0, 1.0), (1.0, 4.0), (4.0, 16.0)]   # band 0: Laplace (k = 0)


def fine_rule(t_max=60.0, panels=100, q=16):
    x, w = np.polynomial.legendre.leggauss(q)
    edges = np.concatenate([[0.0], np.geomspace(0.01, t_max, panels)])
    ts, ws = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        ts.append(0.5 * (b - a) * x + 0.5 * (b + a))
        ws.append(0.5 * (b - a) * w)
    return np.concatenate(ts), np.concatenate(ws)


def samples(seed, n_rand=300):
    rng = np.random.default_rng(seed)
    zz, rr = np.meshgrid(np.linspace(Z_MIN, Z_MAX, 25), np.linspace(0.0, RHO_MAX, 33))
    z = np.concatenate([zz.ravel(), rng.uniform(Z_MIN, Z_MAX, n_rand)])
    rho = np.concatenate([rr.ravel(), rng.uniform(0.0, RHO_MAX, n_rand)])
    return z, rho


def band_kappas(band, n=12):
    k0, k1 = band
    return np.array([k0]) if k1 <= k0 else np.linspace(k0, k1, n)


def design_nodes(band, t, w, z, rho):
    r = np.sqrt(z * z + rho * rho)
    blocks, rhs = [], []
    for k in band_kappas(band):
        s = np.sqrt(t * t + 2.0 * k * t)
        a = np.exp(-np.outer(z, k + t)) * sp.j0(np.outer(rho, s))
        blocks.append(a * r[:, None])                     # error measured in units of 1/r
        rhs.append(np.exp(-k * r))
    A = np.vstack(blocks)
    b = np.concatenate(rhs)
    _, _, piv = la.qr(A * w, pivoting=True, mode="economic")
    for n in range(4, A.shape[1]):
        sel = np.sort(piv[:n])
        wk, *_ = la.lstsq(A[:, sel], b)
        if np.max(np.abs(A[:, sel] @ wk - b)) < 0.5 * EPS:
            return t[sel], wk
    raise RuntimeError("no quadrature found for band %s" % (band,))


def trapezoid_count(tk, wk, band, n_nodes):
    """Smallest even M with the weighted trapezoid error of J0 below 4 EPS / n of the smallest
    1/r (per-node bounds that do not add up coherently; the final check bounds the sum)."""
    rho = np.linspace(0.0, RHO_MAX, 400)
    inv_r_min = 1.0 / np.sqrt(Z_MAX ** 2 + RHO_MAX ** 2)
    for m in range(2, 1000, 2):
        a = 2.0 * np.pi * (np.arange(m) + 0.5) / m
        worst = 0.0
        for k in band_kappas(band, 6):
            s = np.sqrt(tk * tk + 2.0 * k * tk)
            approx = np.cos(s * np.outer(rho, np.cos(a))).mean(axis=1)
            err = np.max(np.abs(approx - sp.j0(s * rho))) * abs(wk) * np.exp(-(k + tk) * Z_MIN)
            worst = max(worst, err)
        if worst < 40.0 * EPS / n_nodes * inv_r_min:
            return m
    raise RuntimeError("trapezoid count not found")


def check(band, ts, ws, ms, seed=7):
    """Largest error of the discrete double sum against the kernel, in units of 1/r, on
    fresh 3-d samples (x, y, z) and kappas of the band."""
    rng = np.random.default_rng(seed)
    n = 400
    z = rng.uniform(Z_MIN, Z_MAX, n)
    ang = rng.uniform(0.0, 2.0 * np.pi, n)
    rho = RHO_MAX * np.sqrt(rng.uniform(0.0, 1.0, n))
    x, y = rho * np.cos(ang), rho * np.sin(ang)
    r = np.sqrt(z * z + rho * rho)
    worst = 0.0
    for k in band_kappas(band, 5):
        acc = np.zeros(n)
        for tk, wk, m in zip(ts, ws, ms):
            s = np.sqrt(tk * tk + 2.0 * k * tk)
            a = 2.0 * np.pi * (np.arange(m // 2) + 0.5) / m             # one of each opposite pair
            ph = s * (np.outer(x, np.cos(a)) + np.outer(y, np.sin(a)))
            acc += wk * np.exp(-(k + tk) * z) * 2.0 * np.cos(ph).sum(axis=1) / m
        worst = max(worst, np.max(np.abs(acc - np.exp(-k * r) / r) * r))
    return worst


def main():
    t, w = fine_rule()
    z, rho = samples(1)
    out = []
    for band in BANDS:
        ts, ws = design_nodes(band, t, w, z, rho)
        ms = [trapezoid_count(tk, wk, band, len(ts)) for tk, wk in zip(ts, ws)]
        err = check(band, ts, ws, ms)
        print("band", band, "nodes", len(ts), "plane waves kept", sum(ms) // 2, "check error", err)
        assert err < EPS, err
        out.append((band, ts, ws, ms, err))
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "pw_quadrature.h"), "w") as f:
        f.write("// Generated by pw_quadrature.py: quadratures of the plane-wave M2L (see there).\n")
        f.write("// Band b covers kappa w in [kPwBandLo[b], kPwBandHi[b]]; band 0 is the Laplace kernel.\n")
        f.write("// Node j of band b: t = kPwT[kPwOff[b] + j], weight kPwW[...], trapezoid count kPwM[...].\n")
        f.write("#pragma once\n\nnamespace afmpb {\n\n")
        f.write("constexpr double kPwEps = %.1e;\n" % EPS)
        f.write("constexpr int kPwBands = %d;\n" % len(out))
        f.write("constexpr double kPwBandLo[kPwBands] = {%s};\n" % ", ".join("%.17g" % b[0][0] for b in out))
        f.write("constexpr double kPwBandHi[kPwBands] = {%s};\n" % ", ".join("%.17g" % b[0][1] for b in out))
        offs = np.cumsum([0] + [len(b[1]) for b in out])
        f.write("constexpr int kPwOff[kPwBands + 1] = {%s};\n" % ", ".join(str(int(o)) for o in offs))
        f.write("constexpr double kPwT[%d] = {\n" % offs[-1])
        for b in out:
            f.write("    %s,\n" % ", ".join("%.17g" % v for v in b[1]))
        f.write("};\nconstexpr double kPwW[%d] = {\n" % offs[-1])
        for b in out:
            f.write("    %s,\n" % ", ".join("%.17g" % v for v in b[2]))
        f.write("};\nconstexpr int kPwM[%d] = {\n" % offs[-1])
        for b in out:
            f.write("    %s,\n" % ", ".join(str(int(v)) for v in b[3]))
        f.write("};\n\n}  // namespace afmpb\n")


if __name__ == "__main__":
    main()
