"""Capsid-scale parity: 60 icosahedral copies of a 20,000-atom globule (10,455,600 nodes,
20,971,440 triangles, 1.2M charges), in the launch configuration the bench times
(precision 1, order 6; the right-hand side and energy by the charge FMM).

The oracle cannot form the whole product or right-hand side at this size, so rows are
sampled and computed one by one: 256 product rows (bar 1e-4 relative L2 over the sample,
the matvec bar) and 256 right-hand-side rows (1e-5 / 2e-5 as for the charge FMM at small
size).  The solve must converge; its true residual is measured with the same FP32
product, whose rounding at 10M nodes is ~1e-5 of ||b||, so the bar on it is 3e-5.  The
charge-FMM energy must agree with the direct sum (a handle built with charge_fmm = 1) to
1e-5.
"""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def capsid():
    return synthetic.capsid()


def test_capsid_product_and_rhs_sampled_rows(capsid):
    import torch
    import paper_1710_06316_gb300 as pb
    mol = capsid
    n = mol.n_nodes
    assert n == 10455600 and len(mol.q) == 1200000
    o = oracle.Oracle.for_molecule(mol)
    x = synthetic.smooth_unknowns(mol.xyz, 2)
    rng = np.random.default_rng(11)
    rows = np.sort(rng.choice(n, 256, replace=False))
    with pb.Handle.for_molecule(mol, order=6, precision=1) as h:
        info = h.info()
        assert info["charge_fmm"] == 1 and info["m2l_rank"] > 0
        xd = torch.tensor(np.asarray(x, np.float32), device="cuda")
        yd = torch.empty_like(xd)
        h.matvec(xd, yd)
        torch.cuda.synchronize()
        y = yd.cpu().numpy().astype(np.float64)
        b = h.rhs()
    y1, y2 = o.matvec_rows(rows, x)
    assert relerr(np.concatenate([y[rows], y[n + rows]]), np.concatenate([y1, y2])) < 1e-4
    b1, b2 = o.rhs_rows(rows, mol.atoms, mol.q)
    assert relerr(b[rows], b1) < 1e-5
    assert relerr(b[n + rows], b2) < 2e-5


def test_capsid_solve_and_energy_fmm_vs_direct(capsid):
    import paper_1710_06316_gb300 as pb
    mol = capsid
    E = {}
    for mode in (2, 1):
        with pb.Handle.for_molecule(mol, order=6, precision=1, charge_fmm=mode) as h:
            f, hh, info = h.solve()
            assert info["status"] == "OK" and info["res_true"] < 3e-5
            E[mode] = h.energy()
    assert abs(E[2] / E[1] - 1) < 1e-5
