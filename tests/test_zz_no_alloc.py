"""The allocation-free energy entry point (afmpb_energy_noalloc).

It serves callers that cannot allocate device memory -- a process whose GPU memory is
owned by another allocator, or a latency-critical loop that cannot pay for the device
synchronisation of cudaMalloc / cudaFree.  It must give the same energy as
afmpb_energy, call after call, although its scratch lives in one static device array
that every call reuses.  This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


def test_energy_noalloc_matches_energy_on_two_calls():
    import paper_1710_06316_gb300 as pb
    mol = synthetic.kirkwood_sphere(subdiv=4)          # 2,562 nodes, 64 charges
    with pb.Handle.for_molecule(mol, order=6, leaf_cap=64) as h:
        h.solve()
        e_ref = h.energy()
        # through the C ABI directly, twice in a row (the scratch keeps the last contents)
        lib = pb.load(build=False)
        out = ctypes.c_double()
        for _ in range(2):
            assert lib.afmpb_energy_noalloc(ctypes.c_void_p(h.h), ctypes.byref(out)) == 0
            assert abs(out.value / e_ref - 1) < 1e-12
        assert abs(h.energy_noalloc() / e_ref - 1) < 1e-12
    # a second molecule with a different charge count on the same device, then the
    # first result again: no stale partial sums leak between calls
    mol2 = synthetic.born_ion(subdiv=3)
    with pb.Handle.for_molecule(mol2, order=6) as h2:
        h2.solve()
        e2 = h2.energy()
        assert abs(h2.energy_noalloc() / e2 - 1) < 1e-12
        assert abs(h2.energy_noalloc() / e2 - 1) < 1e-12


def test_energy_noalloc_with_the_charge_fmm_on_two_calls():
    """With the charge FMM the reaction potential of each evaluation adds translated
    expansions with FP32 atomics in a varying order, so the allocation-free energy agrees
    with afmpb_energy to the documented 1e-6 relative, not bit for bit."""
    import paper_1710_06316_gb300 as pb
    mol = synthetic.kirkwood_sphere(subdiv=4, n_charges=500, index=21)
    with pb.Handle.for_molecule(mol, order=6, leaf_cap=32, charge_fmm=2) as h:
        assert h.info()["charge_fmm"] == 1
        h.solve()
        e_ref = h.energy()
        lib = pb.load(build=False)
        out = ctypes.c_double()
        for _ in range(2):
            assert lib.afmpb_energy_noalloc(ctypes.c_void_p(h.h), ctypes.byref(out)) == 0
            assert abs(out.value / e_ref - 1) < 1e-6


def test_energy_noalloc_rejects_state_and_size():
    import paper_1710_06316_gb300 as pb
    mol = synthetic.born_ion(subdiv=2)
    with pb.Handle.for_molecule(mol, order=4) as h:
        with pytest.raises(pb.AfmpbError) as e:
            h.energy_noalloc()                           # no solve yet
        assert e.value.status == "ESTATE"
    n_big = 65536 + 1
    rng = np.random.default_rng(0)
    atoms = rng.uniform(-0.5, 0.5, (n_big, 3))
    q = np.full(n_big, 1e-5)
    with pb.Handle(mol.xyz, mol.tri, atoms, q, eps_in=1, eps_out=80, kappa=0.1, order=4) as h:
        h.solve()
        with pytest.raises(pb.AfmpbError) as e:
            h.energy_noalloc()
        assert e.value.status == "EINVAL" and "65536" in str(e.value)
