"""Charge-surface sums by FMM (afmpb_options.charge_fmm): the right-hand side of Eq. 5
(charges -> nodes) and the reaction potential of the energy (nodes -> charges) by a
Laplace FMM over one octree holding both point sets, against the FP64 oracle and the
direct-summation kernels.

Bars: right-hand side 1e-5 (potential row) and 2e-5 (normal-derivative row) relative L2
against the oracle.  The charges have both signs, so each node's sum is ~20x smaller than
the sum of its terms' magnitudes and the FMM's truncation error (order 8, ~1e-6 of the
term scale for the potential, more for its derivative, which differentiates the
interpolant) is amplified by that factor.  Energy: 1e-5 against the direct energy, and
the whole solve + energy 1e-4 against the oracle.  Two evaluations of the FMM energy agree
to 1e-6, not bit for bit: the M2L adds into the local expansions with atomics.
"""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def many_charges():
    # 10,242 nodes, 3,000 charges uniform in r < 16 A: several tree levels on both sets
    return synthetic.kirkwood_sphere(subdiv=5, n_charges=3000, index=21)


@pytest.mark.parametrize("precision", [0, 1])
def test_rhs_by_fmm_matches_oracle(many_charges, precision):
    import paper_1710_06316_gb300 as pb
    mol = many_charges
    b_ref = oracle.Oracle.for_molecule(mol).rhs(mol.atoms, mol.q)
    n = mol.n_nodes
    with pb.Handle.for_molecule(mol, order=6, leaf_cap=32, precision=precision, charge_fmm=2) as h:
        info = h.info()
        assert info["charge_fmm"] == 1 and info["charge_fmm_boxes"] > 0
        b = h.rhs()
    assert relerr(b[:n], b_ref[:n]) < 1e-5
    assert relerr(b[n:], b_ref[n:]) < 2e-5
    with pb.Handle.for_molecule(mol, order=6, leaf_cap=32, precision=precision, charge_fmm=1) as h:
        assert h.info()["charge_fmm"] == 0
        b_dir = h.rhs()
    assert relerr(b[:n], b_dir[:n]) < 1e-5 and relerr(b[n:], b_dir[n:]) < 2e-5


def test_energy_by_fmm_matches_direct_and_oracle(many_charges):
    import paper_1710_06316_gb300 as pb
    mol = many_charges
    res = {}
    for mode in (1, 2):
        with pb.Handle.for_molecule(mol, order=6, leaf_cap=32, precision=1, charge_fmm=mode) as h:
            f, hh, info = h.solve()
            assert info["status"] == "OK"
            res[mode] = (np.concatenate([f, hh]), h.energy(), h.energy_noalloc())
    # the FMM energy of the same kind of solution agrees with the direct sum
    assert abs(res[2][1] / res[1][1] - 1) < 1e-5
    assert res[2][2] == pytest.approx(res[2][1], rel=1e-6)
    ref = oracle.Oracle.for_molecule(mol).solve(mol.atoms, mol.q)
    x0 = np.concatenate([ref["f"], ref["h"]])
    assert relerr(res[2][0], x0) < 1e-4
    assert abs(res[2][1] / ref["energy"] - 1) < 1e-4


def test_charge_fmm_auto_threshold_keeps_small_systems_direct():
    import paper_1710_06316_gb300 as pb
    mol = synthetic.born_ion()
    with pb.Handle.for_molecule(mol, order=6) as h:
        assert h.info()["charge_fmm"] == 0
