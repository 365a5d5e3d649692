"""A bounded device wait that expired is reported by every product entry point.

The tensor-core translation kernels give up on a device wait after a fixed number of
polls and set the handle's wait flag instead of hanging the GPU.  The flag is latched:
afmpb_matvec_host reports it for its own product, the next afmpb_matvec /
afmpb_matvec_parts / afmpb_solve call reports an earlier product's expiry (queuing
nothing), and afmpb_sync reports it after waiting for the stream; each report clears it.
The expiry here is set from the host (afmpb_inject_wait_expiry), so nothing faults,
traps or hangs the GPU.  After each report the handle works again and its products match
the oracle.
"""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_expired_wait_is_reported_by_every_product_entry_point():
    import torch
    import paper_1710_06316_gb300 as pb
    mol = synthetic.born_ion(subdiv=3)
    orc = oracle.Oracle.for_molecule(mol)
    x = synthetic.random_unknowns(mol.n_nodes, 5)
    y_ref = orc.matvec(x)
    x32 = x.astype(np.float32)
    with pb.Handle.for_molecule(mol, order=6, leaf_cap=32, precision=1) as h:
        # host-buffer product: its own expiry
        h.inject_wait_expiry()
        with pytest.raises(pb.AfmpbError) as e:
            h.matvec_host(x32)
        assert e.value.status == "ETIMEOUT"
        assert relerr(h.matvec_host(x32).astype(np.float64), y_ref) < 1e-4
        # device product: the latched flag fails the next call, which queues nothing
        xd = torch.tensor(x32, device="cuda")
        yd = torch.full_like(xd, 7.0)
        h.inject_wait_expiry()
        with pytest.raises(pb.AfmpbError) as e:
            h.matvec(xd, yd)
        assert e.value.status == "ETIMEOUT"
        torch.cuda.synchronize()
        assert bool((yd == 7.0).all()), "a refused call must not queue a product"
        with pytest.raises(pb.AfmpbError) as e:      # cleared by the report
            h.inject_wait_expiry()
            h.matvec_parts(xd, yd, pb.PART_FAR)
        assert e.value.status == "ETIMEOUT"
        h.matvec(xd, yd)
        h.sync()
        assert relerr(yd.cpu().numpy().astype(np.float64), y_ref) < 1e-4
        # afmpb_sync reports an expiry of queued work once
        h.matvec(xd, yd)
        h.inject_wait_expiry()
        with pytest.raises(pb.AfmpbError) as e:
            h.sync()
        assert e.value.status == "ETIMEOUT"
        h.sync()
        # the solve reports an earlier expiry, then solves normally
        h.inject_wait_expiry()
        with pytest.raises(pb.AfmpbError) as e:
            h.solve()
        assert e.value.status == "ETIMEOUT"
        f, hh, info = h.solve()
        assert info["status"] == "OK"
        E = h.energy()
    ref = orc.solve(mol.atoms, mol.q)
    assert abs(E / ref["energy"] - 1) < 1e-4
