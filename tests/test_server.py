"""Continuous-batching server (afmpb_server_*): admission by device-memory reservation,
overlap of requests on the device, and the same result alone and in a mix.

Host logic (queue, tickets, budget, refusals) runs without a GPU: every admitted request
then fails at its first CUDA call and reports it.  The GPU tests run real solves.
"""
import numpy as np
import pytest

import synthetic


def _pb():
    import paper_1710_06316_gb300 as pb
    return pb


def test_server_host_logic_without_compute():
    """Admission never reserves more than the budget, every ticket completes exactly once,
    and a request larger than the whole budget is refused at submission."""
    pb = _pb()
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("host-only check; the GPU tests cover the same paths with real solves")
    except ImportError:
        pass
    mol = synthetic.born_ion(subdiv=2)
    est = pb.estimate_bytes(mol.n_nodes, 1)
    with pb.Server(bytes_budget=int(2.5 * est), max_slots=3) as s:
        tickets = [s.submit_molecule(mol) for _ in range(6)]
        for t in tickets:
            r = s.wait(t, 120)
            assert r["status"] != "OK" and r["error"]          # no device here
            assert r["bytes_reserved"] == est
            assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
            with pytest.raises(pb.AfmpbError):
                s.poll(t)                                      # handed out once
        info = s.info()
        assert info["completed"] == 6 and info["failed"] == 6 and info["queued"] == 0
        assert info["bytes_high_water"] <= info["bytes_budget"]
        assert 1 <= info["max_running"] <= 2                   # 2.5 reservations fit twice
        big = pb.estimate_bytes(mol.n_nodes, 1, order=8)
        assert big > 2.5 * est
        with pytest.raises(pb.AfmpbError) as e:
            s.submit_molecule(mol, order=8)
        assert e.value.status == "ENOMEM"


def test_batched_server_host_logic_without_compute():
    """A batched server hands out every ticket exactly once and shuts down cleanly when
    setups fail (no device here): the setup counter and the ready list drain."""
    pb = _pb()
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("host-only check; the GPU tests cover the same paths with real solves")
    except ImportError:
        pass
    mol = synthetic.born_ion(subdiv=2)
    est = pb.estimate_bytes(mol.n_nodes, 1)
    with pb.Server(bytes_budget=8 * est, max_slots=3, max_batch=4, solvers=2) as s:
        tickets = [s.submit_molecule(mol) for _ in range(7)]
        for t in tickets:
            r = s.wait(t, 120)
            assert r["status"] != "OK" and r["error"]
        info = s.info()
    assert info["completed"] == 7 and info["failed"] == 7 and info["queued"] == 0
    assert info["batches"] == 0                                # nothing reached the solver
    with pytest.raises(pb.AfmpbError):
        pb.Server(bytes_budget=est, max_slots=2, max_batch=65)
    with pytest.raises(pb.AfmpbError):
        pb.Server(bytes_budget=est, max_slots=2, max_batch=4, solvers=0)


def _mix():
    """Requests of uneven size: Born ions, Kirkwood spheres and small globules."""
    k4 = synthetic.kirkwood_sphere(subdiv=4)
    k5 = synthetic.kirkwood_sphere(subdiv=5, kappa=0.2)
    born = synthetic.born_ion()
    glob = synthetic.globule(n_atoms=40, index=12)
    return [(born, dict(precision=0)), (k5, dict(precision=1)), (glob, dict(precision=0)),
            (k4, dict(precision=1)), (born, dict(precision=1, order=4)), (k5, dict(precision=0)),
            (glob, dict(precision=1)), (k4, dict(precision=0))]


@pytest.mark.gpu
def test_server_results_alone_equal_in_mix():
    """Each request's energy and surface solution are the same when it runs alone (one
    slot) and when it shares the GPU with the others (four slots, all submitted at once).
    The products differ only by the order of floating-point atomics, so the bar is 1e-6
    relative on the energy and 1e-5 on f and h (GMRES stops at 1e-6)."""
    pb = _pb()
    mix = _mix()
    alone = []
    with pb.Server(bytes_budget=64 << 30, max_slots=1) as s:
        for mol, kw in mix:
            r = s.wait(s.submit_molecule(mol, want_solution=True, **kw), 600)
            assert r["status"] == "OK", r["error"]
            alone.append(r)
    with pb.Server(bytes_budget=64 << 30, max_slots=4) as s:
        tickets = [s.submit_molecule(mol, want_solution=True, **kw) for mol, kw in mix]
        mixed = [s.wait(t, 600) for t in tickets]
        info = s.info()
    assert info["max_running"] >= 2, info                      # requests overlapped
    spans = sorted((r["t_admit"], r["t_done"]) for r in mixed)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    for a, m in zip(alone, mixed):
        assert m["status"] == "OK", m["error"]
        assert abs(m["energy"] / a["energy"] - 1) < 1e-6, (a["energy"], m["energy"])
        for key in ("f", "h"):
            err = np.linalg.norm(m[key] - a[key]) / np.linalg.norm(a[key])
            assert err < 1e-5, (key, err)
        assert m["bytes_used"] <= m["bytes_reserved"]


@pytest.mark.gpu
def test_server_admission_limits_overlap_and_reports_failures():
    """With a budget that holds one large request's admission reservation but not two,
    the reservations stay under the budget at every admission, every large and small
    request still completes with the same energy, and an open mesh fails with EMESH
    without disturbing the others."""
    pb = _pb()
    k5 = synthetic.kirkwood_sphere(subdiv=5)
    born = synthetic.born_ion()
    big = pb.estimate_bytes(k5.n_nodes, k5.atoms.shape[0])
    small = pb.estimate_bytes(born.n_nodes, 1)
    budget = big + small + (small // 2)
    open_tri = born.tri[1:]                                    # one triangle removed
    with pb.Server(bytes_budget=budget, max_slots=4) as s:
        t_big = [s.submit_molecule(k5, precision=1) for _ in range(3)]
        t_bad = s.submit(born.xyz, open_tri, born.atoms, born.q, born.eps_in, born.eps_out, born.kappa)
        t_small = [s.submit_molecule(born) for _ in range(3)]
        rb = [s.wait(t, 600) for t in t_big]
        bad = s.wait(t_bad, 600)
        rs = [s.wait(t, 600) for t in t_small]
        info = s.info()
    assert bad["status"] == "EMESH" and bad["error"]
    for r in rb + rs:
        assert r["status"] == "OK", r["error"]
    assert info["bytes_high_water"] <= budget
    e_ref = rb[0]["energy"]
    assert all(abs(r["energy"] / e_ref - 1) < 1e-6 for r in rb)
    assert info["failed"] == 1


@pytest.mark.gpu
def test_batched_server_results_equal_alone():
    """With batched solves (one solver thread, fused P2P and M2L across the set-up
    requests) each request's energy and surface solution equal its lone solve: 1e-6
    relative on the energy, 1e-5 on f and h."""
    pb = _pb()
    mix = _mix()
    alone = []
    with pb.Server(bytes_budget=64 << 30, max_slots=1) as s:
        for mol, kw in mix:
            r = s.wait(s.submit_molecule(mol, want_solution=True, **kw), 600)
            assert r["status"] == "OK", r["error"]
            alone.append(r)
    # four setup slots feed one solver: requests set up during a solve pile up and are
    # solved together
    with pb.Server(bytes_budget=64 << 30, max_slots=4, max_batch=8, solvers=1) as s:
        tickets = [s.submit_molecule(mol, want_solution=True, **kw) for mol, kw in mix]
        batched = [s.wait(t, 600) for t in tickets]
        info = s.info()
    assert info["batches"] >= 1 and info["batched_requests"] == len(mix)
    assert info["max_batch"] >= 2, info                        # requests were solved together
    for a, m in zip(alone, batched):
        assert m["status"] == "OK", m["error"]
        assert abs(m["energy"] / a["energy"] - 1) < 1e-6, (a["energy"], m["energy"])
        for key in ("f", "h"):
            err = np.linalg.norm(m[key] - a[key]) / np.linalg.norm(a[key])
            assert err < 1e-5, (key, err)
        assert m["bytes_used"] <= m["bytes_reserved"]
