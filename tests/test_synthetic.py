"""Synthetic input generators (host only): the icosahedral group, Taubin smoothing and the
capsid stand-in are checked for the properties the workloads rely on."""
import numpy as np

import oracle
import synthetic


def test_icosahedral_rotations_form_the_group():
    R = synthetic.icosahedral_rotations()
    assert R.shape == (60, 3, 3)
    assert np.allclose(np.einsum("gij,gkj->gik", R, R), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(R), 1.0)
    flat = R.reshape(60, 9)
    d = np.linalg.norm(flat[:, None, :] - flat[None, :, :], axis=2)
    assert (d + np.eye(60) * 10).min() > 1e-6                  # all distinct
    # closed under composition: every product is one of the 60
    for a in range(0, 60, 7):
        for b in range(0, 60, 11):
            p = (R[a] @ R[b]).reshape(9)
            assert np.linalg.norm(flat - p, axis=1).min() < 1e-9


def test_taubin_smoothing_keeps_a_valid_closed_mesh():
    xyz, tri = synthetic.icosphere(3, radius=5.0)
    rng = np.random.default_rng(0)
    noisy = xyz + 0.05 * rng.standard_normal(xyz.shape)
    sm = synthetic.taubin_smooth(noisy, tri, 10)
    st, chi, vol = oracle.mesh_check(sm, tri)
    assert st == 0 and chi == 2
    # smoothing moves the noisy points back toward the sphere without shrinking it
    r0 = np.linalg.norm(noisy, axis=1)
    r1 = np.linalg.norm(sm, axis=1)
    assert r1.std() < 0.5 * r0.std()
    assert abs(r1.mean() / 5.0 - 1) < 0.01


def test_small_capsid_copies_are_disjoint_closed_surfaces():
    m = synthetic.capsid(n_atoms=300, copies=12, grid=1.2)
    nb = m.meta["copy_nodes"]
    assert m.n_nodes == 12 * nb and len(m.q) == 12 * 300
    st, chi, vol = oracle.mesh_check(m.xyz, m.tri)
    assert st == 0 and vol > 0
    # every copy is the first one moved rigidly: same edge lengths, centres 250 A out
    t0 = m.tri[: m.n_tris // 12]
    e0 = np.linalg.norm(m.xyz[t0[:, 0]] - m.xyz[t0[:, 1]], axis=1)
    for c in range(1, 12):
        tc = t0 + c * nb
        ec = np.linalg.norm(m.xyz[tc[:, 0]] - m.xyz[tc[:, 1]], axis=1)
        assert np.allclose(ec, e0, rtol=0, atol=1e-9)
    centres = m.xyz.reshape(12, nb, 3).mean(1)
    r = np.linalg.norm(centres, axis=1)
    assert np.all(np.abs(r - 250.0) < 15.0)
    d = np.linalg.norm(centres[:, None] - centres[None], axis=2) + np.eye(12) * 1e9
    assert d.min() > 60.0
