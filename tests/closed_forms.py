"""Closed-form solvation energies used to pin the oracle (independent of it).

* Born ion: a point charge q at the centre of a sphere of radius a,
  E = (K_c q^2 / 2a) [1 / (eps_out (1 + kappa a)) - 1 / eps_in]   (kcal/mol).
* Kirkwood sphere: charges inside a sphere of radius a, series solution of the
  linearized PB equation (interior Laplace, exterior Yukawa):
    E = (K_c/2) sum_ij q_i q_j / (eps_in a) sum_n g_n (r_i r_j / a^2)^n P_n(cos g_ij)
    g_n = (eps_in (n+1) + eps_out rho_n) / (eps_in n - eps_out rho_n),
    rho_n = x k_n'(x)/k_n(x) = n - x R_n, R_n = k_{n+1}/k_n, x = kappa a,
    R_0 = (1 + x)/x,  R_n = 1/R_{n-1} + (2n+1)/x   (k_n modified spherical Bessel),
  and rho_n = -(n+1) at kappa = 0.
The surface values f, h of the same series solution are given node-wise too.
These are the standard textbook solutions; the tests check the series against itself
in two limits (n = 0 is the Born energy with salt; kappa = 0 gives the classical
(n+1)(eps_in - eps_out)/(n eps_in + (n+1) eps_out)).
"""
from __future__ import annotations

import numpy as np
from scipy.special import eval_legendre

K_C = 332.0636


def born_energy(q, a, eps_in, eps_out, kappa):
    return K_C * q * q / (2.0 * a) * (1.0 / (eps_out * (1.0 + kappa * a)) - 1.0 / eps_in)


def born_surface(q, a, eps_out, kappa):
    """Exact exterior potential f and its normal derivative h on the sphere (with the
    1/(4 pi) of G = 1/(4 pi r) kept in the units, like the discrete system)."""
    f = q / (4.0 * np.pi * eps_out * a * (1.0 + kappa * a))
    h = -q / (4.0 * np.pi * eps_out * a * a)
    return f, h


def kirkwood_g(n_max, a, eps_in, eps_out, kappa):
    g = np.zeros(n_max + 1)
    if kappa == 0.0:
        for n in range(n_max + 1):
            rho = -(n + 1.0)
            g[n] = (eps_in * (n + 1) + eps_out * rho) / (eps_in * n - eps_out * rho)
        return g
    x = kappa * a
    R = (1.0 + x) / x
    for n in range(n_max + 1):
        if n > 0:
            R = 1.0 / R + (2 * n + 1) / x
        rho = n - x * R
        g[n] = (eps_in * (n + 1) + eps_out * rho) / (eps_in * n - eps_out * rho)
    return g


def kirkwood_rho(n_max, a, kappa):
    """rho_n = a phi_n'(a) / phi_n(a) for the decaying exterior solution phi_n of order n:
    n - x R_n with the upward ratio recurrence above, or -(n+1) at kappa = 0."""
    if kappa == 0.0:
        return -(np.arange(n_max + 1) + 1.0)
    x = kappa * a
    rho = np.zeros(n_max + 1)
    R = (1.0 + x) / x
    for n in range(n_max + 1):
        if n > 0:
            R = 1.0 / R + (2 * n + 1) / x
        rho[n] = n - x * R
    return rho


def _terms(atoms, a, tol, n_max):
    """Terms of the surface series: its n-th term scales as (r_max / a)^n."""
    r = np.linalg.norm(atoms, axis=1)
    ratio = r.max() / a if r.size else 0.0
    if ratio > 0:
        return min(n_max, int(np.ceil(np.log(tol) / np.log(ratio))) + 2)
    return n_max


def kirkwood_surface(atoms, q, pts, a, eps_in, eps_out, kappa, tol=1e-14, n_max=400):
    """Exact f (potential) and h (exterior normal derivative) at points pts on the sphere
    |x| = a.  With c_n = q_j r_j^n / (4 pi eps_in) the Coulomb part inside is
    c_n r^-(n+1) P_n, the reaction part g_n c_n r^n / a^(2n+1) P_n (the g_n of the energy),
    and continuity at r = a makes the exterior coefficient (1 + g_n) c_n a^-(n+1):
      f = sum_j q_j / (4 pi eps_in a)   sum_n (1 + g_n)       (r_j / a)^n P_n(cos g_j)
      h = sum_j q_j / (4 pi eps_in a^2) sum_n (1 + g_n) rho_n (r_j / a)^n P_n(cos g_j)."""
    atoms = np.asarray(atoms, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    pts = np.asarray(pts, dtype=np.float64)
    n_use = _terms(atoms, a, tol, n_max)
    g = kirkwood_g(n_use, a, eps_in, eps_out, kappa)
    rho = kirkwood_rho(n_use, a, kappa)
    r = np.linalg.norm(atoms, axis=1)
    u = pts / np.linalg.norm(pts, axis=1, keepdims=True)
    with np.errstate(invalid="ignore", divide="ignore"):
        cosg = (u @ atoms.T) / np.maximum(r, 1e-300)[None, :]
    cosg = np.clip(np.where(r[None, :] > 0, cosg, 1.0), -1.0, 1.0)
    f = np.zeros(pts.shape[0])
    h = np.zeros(pts.shape[0])
    for n in range(n_use + 1):
        t = (eval_legendre(n, cosg) * ((r / a) ** n * q)[None, :]).sum(axis=1)
        f += (1.0 + g[n]) * t
        h += (1.0 + g[n]) * rho[n] * t
    return f / (4 * np.pi * eps_in * a), h / (4 * np.pi * eps_in * a * a)


def kirkwood_energy(atoms, q, a, eps_in, eps_out, kappa, tol=1e-14, n_max=400):
    atoms = np.asarray(atoms, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    r = np.linalg.norm(atoms, axis=1)
    rmax = r.max() if r.size else 0.0
    ratio = (rmax / a) ** 2
    n_use = n_max
    if ratio > 0:
        n_use = min(n_max, int(np.ceil(np.log(tol) / np.log(ratio))) + 2)
    g = kirkwood_g(n_use, a, eps_in, eps_out, kappa)
    rr = np.outer(r, r) / (a * a)
    with np.errstate(invalid="ignore", divide="ignore"):
        cosg = (atoms @ atoms.T) / np.outer(np.maximum(r, 1e-300), np.maximum(r, 1e-300))
    cosg = np.clip(np.nan_to_num(cosg, nan=1.0), -1.0, 1.0)
    qq = np.outer(q, q)
    S = np.zeros_like(rr)
    for n in range(n_use + 1):
        S += g[n] * rr ** n * eval_legendre(n, cosg)
    return 0.5 * K_C * float((qq * S).sum()) / (eps_in * a)


def solid_angle(x, a, b, c):
    """Signed solid angle of triangle (a,b,c) seen from x (Van Oosterom & Strackee 1983);
    positive when the triangle is counter-clockwise seen from outside and x is inside."""
    A, B, Cc = a - x, b - x, c - x
    la, lb, lc = np.linalg.norm(A), np.linalg.norm(B), np.linalg.norm(Cc)
    num = np.dot(A, np.cross(B, Cc))
    den = la * lb * lc + np.dot(A, B) * lc + np.dot(A, Cc) * lb + np.dot(B, Cc) * la
    return 2.0 * np.arctan2(num, den)
