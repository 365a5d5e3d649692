"""Leaf-capacity and tile-shape autotuner (AFMPB_LEAF_CAP_AUTO): measured P2P per
candidate tree plus a far-field model calibrated on the handle's own product, then the P2P
resident blocks and work-unit size and the tensor-core M2L item size by timing the kernels
on the finished handle."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_measured_candidate_and_caches_it():
    import paper_1710_06316_gb300 as pb
    mol = synthetic.kirkwood_sphere(subdiv=6)            # 40,962 nodes
    with pb.Handle.for_molecule(mol, order=6, precision=1, leaf_cap=pb.LEAF_CAP_AUTO) as h:
        info = h.info()
        rep = h.autotune()
        assert info["autotuned"] == 1 and rep is not None
        assert rep["n_candidates"] >= 5
        assert rep["best_cap"] in rep["cap"]
        k = rep["cap"].index(rep["best_cap"])
        assert rep["predicted_ms"][k] == min(rep["predicted_ms"])
        assert rep["predicted_best_ms"] <= rep["predicted_start_ms"] + 1e-12
        assert all(t > 0 for t in rep["p2p_ms"])
        # rebuilt at the best capacity only when it predicts a gain of at least 3%
        rebuilt = rep["best_cap"] != rep["start_cap"] and rep["predicted_best_ms"] < 0.97 * rep["predicted_start_ms"]
        assert info["leaf_cap"] == (rep["best_cap"] if rebuilt else rep["start_cap"])
        # tile shapes: chosen among the candidates, never slower than the defaults
        assert rep["p2p_resident"] in (4, 5, 6) and rep["p2p_units_per_block"] in (1, 2, 3, 4, 6)
        assert 0 < rep["p2p_ms_tuned"] <= rep["p2p_ms_default"]
        assert rep["m2l_runs_per_item"] in (0, 8, 16, 24, 32)
        if rep["m2l_runs_per_item"]:
            assert 0 < rep["m2l_ms_tuned"] <= rep["m2l_ms_default"]
        # the product still meets the bar (sampled rows against the oracle)
        o = oracle.Oracle.for_molecule(mol)
        x = synthetic.random_unknowns(mol.n_nodes, 21)
        rows = np.sort(np.random.default_rng(3).choice(mol.n_nodes, 256, replace=False))
        r1, r2 = o.matvec_rows(rows, x)
        import torch
        xd = torch.tensor(x.astype(np.float32), device="cuda")
        yd = torch.empty_like(xd)
        h.matvec(xd, yd)
        torch.cuda.synchronize()
        y = yd.cpu().numpy().astype(np.float64)
        got = np.concatenate([y[rows], y[mol.n_nodes + rows]])
        ref = np.concatenate([r1, r2])
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-4
        chosen = info["leaf_cap"]
    # same size class: no tuning, the cached capacity
    mol2 = synthetic.kirkwood_sphere(subdiv=6, kappa=0.2)
    with pb.Handle.for_molecule(mol2, order=6, precision=1, leaf_cap=pb.LEAF_CAP_AUTO) as h2:
        assert h2.info()["autotuned"] == 0
        assert h2.autotune() is None
        assert h2.info()["leaf_cap"] == rep["best_cap"]
    assert chosen in (rep["best_cap"], rep["start_cap"])
