"""Plane-wave M2L (afmpb_options.m2l_method = 1): the exponential expansions of FMM97 as
an alternative to the dense list-2 translations.

The quadratures (pw_quadrature.h) are pinned to the kernels themselves: the discrete
double sum -- t-nodes and weights, trapezoid rule in the angle -- is evaluated here in
float64 at random well-separated points of every band and compared with exp(-k r)/r; its
error must stay below 1e-6 of 1/r (the bound the generator asks for).  On the GPU the
plane-wave product matches the oracle within the product bar (1e-4), the dense product
without compression within 1e-5 (both are exact kernel sums between the same Chebyshev
expansions, up to 1e-6 of the quadrature), and a plane-wave solve gives the oracle's
energy to 1e-4.
"""
import os
import re

import numpy as np
import pytest

import oracle
import synthetic

HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_1710_06316_gb300", "csrc", "pw_quadrature.h")


def _tables():
    txt = open(HEADER).read()

    def arr(name, conv=float):
        m = re.search(r"%s\[[^\]]*\]\s*=\s*\{([^}]*)\}" % name, txt)
        return np.array([conv(v) for v in m.group(1).replace("\n", " ").split(",") if v.strip()])

    return (arr("kPwBandLo"), arr("kPwBandHi"), arr("kPwOff", int), arr("kPwT"), arr("kPwW"), arr("kPwM", int))


def _discrete(k, ts, ws, ms, x, y, z):
    acc = np.zeros_like(z)
    for t, w, m in zip(ts, ws, ms):
        s = np.sqrt(t * t + 2.0 * k * t)
        a = 2.0 * np.pi * (np.arange(m // 2) + 0.5) / m
        ph = s * (np.outer(x, np.cos(a)) + np.outer(y, np.sin(a)))
        acc += w * np.exp(-(k + t) * z) * 2.0 * np.cos(ph).sum(axis=1) / m
    return acc


def test_quadratures_reproduce_the_kernels():
    lo, hi, off, T, W, M = _tables()
    assert len(lo) == 4 and lo[0] == hi[0] == 0.0                      # band 0: Laplace
    assert np.all(M % 2 == 0) and np.all(T > 0)
    rng = np.random.default_rng(3)
    n = 2000
    # separations of well-separated boxes in box units: along the axis 1..4, across <= 4 sqrt 2
    z = rng.uniform(1.0, 4.0, n)
    x = rng.uniform(-4.0, 4.0, n)
    y = rng.uniform(-4.0, 4.0, n)
    r = np.sqrt(x * x + y * y + z * z)
    for b in range(len(lo)):
        sl = slice(off[b], off[b + 1])
        for k in sorted({lo[b], hi[b], 0.5 * (lo[b] + hi[b])}):
            got = _discrete(k, T[sl], W[sl], M[sl], x, y, z)
            err = np.max(np.abs(got - np.exp(-k * r) / r) * r)
            assert err < 1e-6, (b, k, err)


def test_a_wrong_weight_or_node_is_caught():
    """The pin is sensitive: one weight off by 1e-4 relative, or one node moved by 1e-4,
    breaks the bound."""
    lo, hi, off, T, W, M = _tables()
    rng = np.random.default_rng(4)
    z = rng.uniform(1.0, 4.0, 500)
    x = rng.uniform(-4.0, 4.0, 500)
    y = rng.uniform(-4.0, 4.0, 500)
    r = np.sqrt(x * x + y * y + z * z)
    sl = slice(off[0], off[1])
    Ts, Ws = T[sl].copy(), W[sl].copy()
    Ws[3] *= 1.0 + 1e-4
    assert np.max(np.abs(_discrete(0.0, Ts, Ws, M[sl], x, y, z) - 1 / r) * r) > 1e-6
    Ts, Ws = T[sl].copy(), W[sl].copy()
    Ts[5] *= 1.0 + 1e-4
    assert np.max(np.abs(_discrete(0.0, Ts, Ws, M[sl], x, y, z) - 1 / r) * r) > 1e-6


def _gpu_matvec(h, x):
    import torch
    xd = torch.tensor(x.astype(np.float32), device="cuda")
    yd = torch.empty_like(xd)
    h.matvec(xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.gpu
@pytest.mark.parametrize("which", ["born", "kirkwood_k0.3", "globule"])
def test_plane_wave_product_matches_oracle_and_dense(which):
    import paper_1710_06316_gb300 as pb
    mol = {"born": lambda: synthetic.born_ion(),
           "kirkwood_k0.3": lambda: synthetic.kirkwood_sphere(subdiv=5, kappa=0.3),
           "globule": lambda: synthetic.globule(n_atoms=200, index=3)}[which]()
    x = synthetic.random_unknowns(mol.n_nodes, 11)
    y_ref = oracle.Oracle.for_molecule(mol).matvec(x)
    with pb.Handle.for_molecule(mol, order=6, precision=0, m2l_method=1) as h:
        assert h.info()["n_m2l_pairs"] > 0
        y_pw = _gpu_matvec(h, x)
    with pb.Handle.for_molecule(mol, order=6, precision=0, m2l_tol=-1.0) as h:
        y_dense = _gpu_matvec(h, x)
    assert _rel(y_pw, y_ref) < 1e-4
    assert _rel(y_pw, y_dense) < 1e-5


@pytest.mark.gpu
def test_plane_wave_solve_and_energy():
    import paper_1710_06316_gb300 as pb
    mol = synthetic.born_ion()
    ref = oracle.Oracle.for_molecule(mol).solve(mol.atoms, mol.q)
    with pb.Handle.for_molecule(mol, order=6, precision=0, m2l_method=1) as h:
        f, hh, info = h.solve()
        E = h.energy()
    assert info["status"] == "OK"
    assert _rel(np.concatenate([f, hh]), np.concatenate([ref["f"], ref["h"]])) < 1e-4
    assert abs(E / ref["energy"] - 1) < 1e-4


@pytest.mark.gpu
@pytest.mark.parametrize("order,kappa", [(4, 0.104), (8, 0.104), (6, 0.0)])
def test_plane_wave_orders_and_laplace_only(order, kappa):
    """Other expansion orders (4, 8: the tables and index maps are per order) and kappa = 0
    (only the Laplace band) against the dense product without compression."""
    import paper_1710_06316_gb300 as pb
    mol = synthetic.kirkwood_sphere(subdiv=4, kappa=kappa)
    x = synthetic.random_unknowns(mol.n_nodes, 17)
    with pb.Handle.for_molecule(mol, order=order, precision=0, m2l_method=1, leaf_cap=32) as h:
        assert h.info()["n_m2l_pairs"] > 0
        y_pw = _gpu_matvec(h, x)
    with pb.Handle.for_molecule(mol, order=order, precision=0, m2l_tol=-1.0, leaf_cap=32) as h:
        y_dense = _gpu_matvec(h, x)
    assert _rel(y_pw, y_dense) < 1e-5
