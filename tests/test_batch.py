"""Batched solve (afmpb_solve_batch): several problems' GMRES in lockstep with one fused
P2P launch and one fused tensor-core M2L launch per Arnoldi step.

Each problem keeps its own arithmetic: the batch changes only which launch does its work
and the order of floating-point atomic additions.  So a problem solved in a batch matches
the same problem solved alone to 1e-6 on the energy and 1e-5 on the surface solution (the
GMRES tolerance is 1e-6), takes the same number of Arnoldi steps (one more or less where a
residual sits at the tolerance), and the small ones match the oracle's dense solve to
1e-4, the bar of the single-problem parity tests.
"""
import numpy as np
import pytest

import oracle
import synthetic


def _pb():
    import paper_1710_06316_gb300 as pb
    return pb


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _uneven_eight():
    """Eight requests of uneven size and screening: Born ions, Kirkwood spheres of two
    sizes and kappas, and small globules (2.5k to 41k nodes)."""
    born = synthetic.born_ion()
    born_k = synthetic.born_ion(subdiv=3, kappa=0.3)
    k4 = synthetic.kirkwood_sphere(subdiv=4)
    k5 = synthetic.kirkwood_sphere(subdiv=5, kappa=0.2)
    k5b = synthetic.kirkwood_sphere(subdiv=5, radius=14.0, kappa=0.05)
    glob = synthetic.globule(n_atoms=40, index=12)
    glob2 = synthetic.globule(n_atoms=120, index=5)
    return [born, k5, glob, k4, born_k, k5b, glob2, k4]


def _solve_alone(pb, mol, **kw):
    with pb.Handle.for_molecule(mol, **kw) as h:
        f, hh, info = h.solve()
        return f, hh, info, h.energy()


def _check_against_alone(pb, mols, kws):
    alone = [_solve_alone(pb, m, **kw) for m, kw in zip(mols, kws)]
    hs = [pb.Handle.for_molecule(m, **kw) for m, kw in zip(mols, kws)]
    try:
        out = pb.solve_batch(hs)
        energies = [h.energy() for h in hs]
    finally:
        for h in hs:
            h.close()
    for (f, hh, info), E, (fa, ha, ia, Ea) in zip(out, energies, alone):
        assert info["status"] == "OK"
        assert abs(E / Ea - 1) < 1e-6, (E, Ea)
        x, xa = np.concatenate([f, hh]), np.concatenate([fa, ha])
        assert relerr(x, xa) < 1e-5
        assert abs(info["iters"] - ia["iters"]) <= 1, (info["iters"], ia["iters"])
        assert info["res_true"] < 1e-5
    return out, energies


@pytest.mark.gpu
def test_batch_of_eight_uneven_requests_matches_alone_and_oracle():
    """Mixed precision, one compressed rank: P2P and M2L both fused across the eight."""
    pb = _pb()
    mols = _uneven_eight()
    kws = [dict(order=6, precision=1)] * len(mols)
    out, energies = _check_against_alone(pb, mols, kws)
    # the small ones against the oracle's dense solve
    for i in (0, 2, 4):
        mol = mols[i]
        ref = oracle.Oracle.for_molecule(mol).solve(mol.atoms, mol.q)
        f, hh, _ = out[i]
        assert relerr(np.concatenate([f, hh]), np.concatenate([ref["f"], ref["h"]])) < 1e-4
        assert abs(energies[i] / ref["energy"] - 1) < 1e-4


@pytest.mark.gpu
def test_batch_mixed_precisions_and_orders():
    """Plain FP32 and mixed problems, orders 4 and 6: P2P fused, each M2L in its own chain."""
    pb = _pb()
    born = synthetic.born_ion()
    k4 = synthetic.kirkwood_sphere(subdiv=4)
    glob = synthetic.globule(n_atoms=40, index=12)
    mols = [born, k4, glob, k4]
    kws = [dict(order=6, precision=0), dict(order=6, precision=1), dict(order=4, precision=0),
           dict(order=6, precision=0, orth=0)]
    _check_against_alone(pb, mols, kws)


@pytest.mark.gpu
def test_batch_restarts_and_repeat():
    """Short restart cycles (restart 8) force several cycles with problems stopping in
    different ones; a second batched solve of the same handles gives the same answer."""
    pb = _pb()
    mols = [synthetic.kirkwood_sphere(subdiv=4), synthetic.born_ion(), synthetic.globule(n_atoms=40, index=12)]
    kws = [dict(order=6, precision=1, restart=8, max_restart=60)] * 3
    _check_against_alone(pb, mols, kws)
    hs = [pb.Handle.for_molecule(m, **kw) for m, kw in zip(mols, kws)]
    try:
        a = pb.solve_batch(hs)
        ea = [h.energy() for h in hs]
        b = pb.solve_batch(hs)
        eb = [h.energy() for h in hs]
    finally:
        for h in hs:
            h.close()
    for (fa, ha, ia), (fb, hb, ib), x, y in zip(a, b, ea, eb):
        assert ia["restarts"] >= 1 or ia["iters"] <= 8
        assert abs(x / y - 1) < 1e-6
        assert relerr(np.concatenate([fb, hb]), np.concatenate([fa, ha])) < 1e-5


@pytest.mark.gpu
def test_batch_rejects_bad_batches():
    pb = _pb()
    born = synthetic.born_ion()
    with pb.Handle.for_molecule(born) as h:
        with pytest.raises(pb.AfmpbError) as e:
            pb.solve_batch([h, h])
        assert e.value.status == "EINVAL"
    with pb.Handle(born.xyz, born.tri, None, None, born.eps_in, born.eps_out, born.kappa) as h0, \
            pb.Handle.for_molecule(born) as h1:
        with pytest.raises(pb.AfmpbError) as e:
            pb.solve_batch([h1, h0])
        assert e.value.status == "ESTATE"


@pytest.mark.gpu
def test_batch_of_one_and_per_problem_statuses():
    """A batch of one equals the lone solve; a problem that cannot converge within its
    restart budget reports ENOCONV while the others of the batch still reach OK."""
    pb = _pb()
    born = synthetic.born_ion()
    k4 = synthetic.kirkwood_sphere(subdiv=4)
    f1, h1, i1, E1 = _solve_alone(pb, born, order=6, precision=1)
    with pb.Handle.for_molecule(born, order=6, precision=1) as h:
        [(f, hh, info)] = pb.solve_batch([h])
        E = h.energy()
    assert info["status"] == "OK" and abs(E / E1 - 1) < 1e-6
    assert relerr(np.concatenate([f, hh]), np.concatenate([f1, h1])) < 1e-5
    hs = [pb.Handle.for_molecule(born, order=6, precision=1),
          pb.Handle.for_molecule(k4, order=6, precision=1, restart=2, max_restart=1),   # cannot reach 1e-6
          pb.Handle.for_molecule(k4, order=6, precision=1)]
    try:
        out = pb.solve_batch(hs, raise_on_noconv=False)
    finally:
        for h in hs:
            h.close()
    assert [o[2]["status"] for o in out] == ["OK", "ENOCONV", "OK"]
    assert out[1][2]["restarts"] == 1 and out[1][2]["iters"] <= 4
