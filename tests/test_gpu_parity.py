"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars (floating point, FP32 GPU arithmetic against the FP64 oracle):
* geometry (computed in FP64 on the device): 1e-12 relative;
* near-field coefficients (FP32 quadrature on target-relative geometry): 1e-5 of the
  largest coefficient (rounding of sums over up to ~1e4 quadrature points);
* products: relative L2 error <= 1e-4 on the whole vector and on each block (the bar
  the matvec must meet at the configured FMM order);
* right-hand side: 1e-5; GMRES solution and solvation energy: 1e-4.
Integer work (near-set membership, tree lists) is compared exactly or checked for
validity where several answers are correct.
"""
import numpy as np
import pytest

import oracle
import synthetic
from closed_forms import born_energy

pytestmark = pytest.mark.gpu

TOL_MATVEC = 1e-4


def torch_cuda():
    import torch
    return torch


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_matvec(h, x, parts=7):
    torch = torch_cuda()
    xd = torch.tensor(np.asarray(x, np.float32), device="cuda")
    yd = torch.empty_like(xd)
    h.matvec_parts(xd, yd, parts)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def born():
    import paper_1710_06316_gb300 as pb
    mol = synthetic.born_ion()          # 2,562 nodes, order 6
    h = pb.Handle.for_molecule(mol, order=6, tol=1e-6)
    o = oracle.Oracle.for_molecule(mol)
    yield mol, h, o
    h.close()


def test_geometry_matches_oracle(born):
    mol, h, o = born
    a, n, r = h.geometry()
    a0, n0, r0 = o.geometry()
    np.testing.assert_allclose(a, a0, rtol=1e-12)
    np.testing.assert_allclose(n, n0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r, r0, rtol=1e-12)


def test_near_set_and_coefficients_match_oracle(born):
    mol, h, o = born
    rp, col, coef, whole = h.near()
    rp0, col0, coef0 = o.near_csr()
    n = mol.n_nodes
    assert rp[-1] == rp0[-1]
    for p in range(n):
        g = np.sort(col[rp[p]:rp[p + 1]])
        assert np.array_equal(g, col0[rp0[p]:rp0[p + 1]]), p
    # coefficients: near - far, or the whole near value for the self entry and for the
    # close pairs the P2P pass leaves out (FP32 distance <= 0.9 c (rho_p + rho_t))
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert whole[rows == col].all()
    _, _, rho = o.geometry()
    dist = np.linalg.norm(mol.xyz[rows] - mol.xyz[col], axis=1)
    lim = 0.9 * 2.0 * (rho[rows] + rho[col])
    assert (dist[whole] <= lim[whole] * (1 + 1e-5)).all()
    assert whole[rows != col].any()
    near = o.coeffs(rows, col, rule=o.NEAR)
    far = o.coeffs(rows, col, rule=o.FAR)
    ref = np.where(whole[:, None], near, near - far)
    scale = np.abs(ref).max(axis=0)
    err = np.abs(coef - ref).max(axis=0) / scale
    # FP32 quadrature over up to ~1e4 points: rounding ~ sqrt(1e4) * 2^-24 ~ 1e-5
    assert err.max() < 1e-5, err


def test_near_set_and_coefficients_match_oracle_on_sliver_globule(small_globule):
    """The near set and its coefficients on the raw isosurface of a small globule (sliver
    triangles kept): exactly the oracle's set on every row; coefficients on 300 sampled
    rows.  The double-layer and derivative blocks (dB, dC, dD) meet the Born check's 1e-5
    of the largest; the single-layer block dA reaches 7e-5 on this mesh (FP32 quadrature
    near sliver patches, measured), so its bar here is 1e-4 -- the product bar, which the
    full product on the same mesh meets."""
    import paper_1710_06316_gb300 as pb
    mol, o, _, _ = small_globule
    with pb.Handle.for_molecule(mol, order=6, leaf_cap=64) as h:
        rp, col, coef, whole = h.near()
    rp0, col0, _ = o.near_csr()
    n = mol.n_nodes
    assert rp[-1] == rp0[-1]
    for p in range(n):
        assert np.array_equal(np.sort(col[rp[p]:rp[p + 1]]), col0[rp0[p]:rp0[p + 1]]), p
    sel = np.sort(np.random.default_rng(9).choice(n, 300, replace=False))
    ent = np.concatenate([np.arange(rp[p], rp[p + 1]) for p in sel])
    rows = np.repeat(np.arange(n), np.diff(rp))[ent]
    cols = col[ent]
    near = o.coeffs(rows, cols, rule=o.NEAR)
    far = o.coeffs(rows, cols, rule=o.FAR)
    ref = np.where(whole[ent][:, None], near, near - far)
    err = np.abs(coef[ent] - ref).max(axis=0) / np.abs(ref).max(axis=0)
    assert err[0] < 1e-4 and err[1:].max() < 1e-5, err


def test_tree_lists_cover_every_pair_once(born):
    mol, h, o = born
    check_tree_coverage(h)


def check_tree_coverage(h):
    t = h.tree()
    nb = len(t["level"])
    n = h.n
    children = [[] for _ in range(nb)]
    for b in range(nb):
        if t["parent"][b] >= 0:
            children[t["parent"][b]].append(b)
    leaves = [b for b in range(nb) if not children[b]]
    rng = t["range"]
    # leaves tile [0, n)
    cover = np.zeros(n, int)
    for b in leaves:
        cover[rng[b, 0]:rng[b, 1]] += 1
    assert np.all(cover == 1)
    anc = t["anchor"]
    lev = t["level"]

    def adjacent(a, b):
        if lev[a] > lev[b]:
            a, b = b, a
        s = lev[b] - lev[a]
        lo = anc[a] << s
        hi = (anc[a] + 1) << s
        return bool(np.all(anc[b] + 1 >= lo) and np.all(anc[b] <= hi))

    for T in leaves:
        cnt = np.zeros(n, int)
        for c in list(t["u_idx"][t["u_ptr"][T]:t["u_ptr"][T + 1]]):
            assert adjacent(T, c) and not children[c]
            cnt[rng[c, 0]:rng[c, 1]] += 1
        for c in t["w_idx"][t["w_ptr"][T]:t["w_ptr"][T + 1]]:
            assert not adjacent(T, c) and adjacent(T, t["parent"][c])
            cnt[rng[c, 0]:rng[c, 1]] += 1
        A = T
        while A >= 0:
            for c in t["v_idx"][t["v_ptr"][A]:t["v_ptr"][A + 1]]:
                assert lev[c] == lev[A] and np.abs(anc[c] - anc[A]).max() >= 2
                cnt[rng[c, 0]:rng[c, 1]] += 1
            for c in t["x_idx"][t["x_ptr"][A]:t["x_ptr"][A + 1]]:
                assert not children[c] and not adjacent(A, c)
                cnt[rng[c, 0]:rng[c, 1]] += 1
            A = t["parent"][A]
        assert np.all(cnt == 1), (T, np.unique(cnt))


def skipped_far_rule(h, o, x):
    """The oracle's far-rule terms of the pairs (t != p) whose near entry is whole."""
    n = h.n
    rp, col, _, whole = h.near()
    rows = np.repeat(np.arange(n), np.diff(rp))
    sel = whole & (rows != col)
    p, t = rows[sel], col[sel].astype(np.int64)
    far = o.coeffs(p, t, rule=o.FAR)
    f, hh = x[:n], x[n:]
    out = np.zeros(2 * n)
    np.add.at(out, p, far[:, 1] * f[t] - far[:, 0] * hh[t])
    np.add.at(out, n + p, far[:, 3] * f[t] - far[:, 2] * hh[t])
    return out


@pytest.mark.parametrize("kind", ["smooth", "random"])
def test_matvec_matches_oracle_born(born, kind):
    mol, h, o = born
    n = mol.n_nodes
    x = synthetic.smooth_unknowns(mol.xyz, 0) if kind == "smooth" else synthetic.random_unknowns(n, 0)
    y_ref = o.matvec(x)
    y = gpu_matvec(h, x)
    assert relerr(y, y_ref) < TOL_MATVEC
    assert relerr(y[:n], y_ref[:n]) < TOL_MATVEC
    assert relerr(y[n:], y_ref[n:]) < TOL_MATVEC
    # parts: point sums alone (FMM + P2P) against the oracle's far rule over all t != p,
    # less the close pairs that the P2P pass leaves to the near CSR (its `whole` entries,
    # each checked against the skip radius in the near-set test)
    y_pt = gpu_matvec(h, x, parts=1 | 2)
    y_pt_ref = o.matvec(x, mode=1) - skipped_far_rule(h, o, x)
    assert relerr(y_pt, y_pt_ref) < TOL_MATVEC
    # near correction alone
    y_nr = gpu_matvec(h, x, parts=4)
    assert relerr(y_nr, y_ref - y_pt_ref) < 1e-5


def test_matvec_host_buffers_equal_device_buffers(born):
    """Same product through host buffers.  M2L accumulates with float atomics, so two
    products agree to FP32 rounding, not bit for bit."""
    mol, h, o = born
    x = synthetic.random_unknowns(mol.n_nodes, 3).astype(np.float32)
    y_dev = gpu_matvec(h, x)
    y_host = h.matvec_host(x).astype(np.float64)
    assert relerr(y_host, y_dev) < 1e-6
    np.testing.assert_allclose(y_host, y_dev, rtol=0, atol=2e-5 * np.abs(y_dev).max())


def test_rhs_matches_oracle(born):
    mol, h, o = born
    np.testing.assert_allclose(h.rhs(), o.rhs(mol.atoms, mol.q), rtol=1e-5)


def test_solve_and_energy_match_oracle_and_born(born):
    mol, h, o = born
    f, hh, info = h.solve()
    assert info["status"] == "OK"
    ref = o.solve(mol.atoms, mol.q)
    x = np.concatenate([f, hh])
    x0 = np.concatenate([ref["f"], ref["h"]])
    assert relerr(x, x0) < 1e-4
    E = h.energy()
    assert abs(E / ref["energy"] - 1) < 1e-4
    E_born = born_energy(1.0, 2.0, 1.0, 80.0, 0.104)
    assert abs(E / E_born - 1) < 0.005
    assert info["res_true"] < 1e-5


@pytest.mark.parametrize("order", [4, 6, 8])
@pytest.mark.parametrize("kappa", [0.0, 0.5])
def test_matvec_orders_and_kappa_kirkwood_small(order, kappa):
    """Kirkwood geometry at subdivision 5 (10,242 nodes, several tree levels, ragged
    leaves) with off-centre charges; full comparison against the oracle."""
    import paper_1710_06316_gb300 as pb
    mol = synthetic.kirkwood_sphere(subdiv=5, kappa=kappa)
    o = oracle.Oracle.for_molecule(mol)
    x = synthetic.random_unknowns(mol.n_nodes, 5)
    with pb.Handle.for_molecule(mol, order=order, leaf_cap=32) as h:
        assert h.info()["n_m2l_pairs"] > 0
        y = gpu_matvec(h, x)
    y_ref = o.matvec(x)
    bar = {4: 1e-3, 6: TOL_MATVEC, 8: TOL_MATVEC}[order]
    assert relerr(y, y_ref) < bar


@pytest.mark.parametrize("kappa", [0.0, 0.104])
def test_mixed_precision_tensor_core_m2l(kappa):
    """precision 1: M2L on the tensor cores (BF16 hi/lo split, FP32 accumulation) must
    meet the same bar against the oracle and stay within 1e-5 of the FP32 product (the
    split keeps about 16 mantissa bits per translation product)."""
    import paper_1710_06316_gb300 as pb
    mol = synthetic.kirkwood_sphere(subdiv=5, kappa=kappa)
    o = oracle.Oracle.for_molecule(mol)
    x = synthetic.random_unknowns(mol.n_nodes, 9)
    with pb.Handle.for_molecule(mol, order=6, leaf_cap=32, precision=1) as h:
        assert h.info()["n_m2l_pairs"] > 0 and h.info()["precision"] == 1
        y_tc = gpu_matvec(h, x)
    with pb.Handle.for_molecule(mol, order=6, leaf_cap=32, precision=0) as h:
        y_fp = gpu_matvec(h, x)
    y_ref = o.matvec(x)
    assert relerr(y_tc, y_ref) < TOL_MATVEC
    assert relerr(y_tc, y_fp) < 1e-5


@pytest.mark.parametrize("precision", [0, 1])
def test_m2l_compression_against_full_translations(precision):
    """Compressed list-2 translations (the singular vectors of the stacked translation
    matrices above m2l_tol): the rank grows as the cutoff falls, every setting meets the
    oracle bar, and at 1e-6 the product agrees with the full n^3 translations to 1e-5."""
    import paper_1710_06316_gb300 as pb
    mol = synthetic.kirkwood_sphere(subdiv=5, kappa=0.104)
    o = oracle.Oracle.for_molecule(mol)
    x = synthetic.random_unknowns(mol.n_nodes, 11)
    y_ref = o.matvec(x)
    res = {}
    for tol in (-1.0, 1e-4, 1e-6):
        with pb.Handle.for_molecule(mol, order=6, leaf_cap=32, precision=precision, m2l_tol=tol) as h:
            assert h.info()["n_m2l_pairs"] > 0
            res[tol] = (h.info()["m2l_rank"], gpu_matvec(h, x))
    assert res[-1.0][0] == 0
    assert 0 < res[1e-4][0] <= res[1e-6][0] < 216
    assert res[1e-4][0] % 16 == 0 and res[1e-6][0] % 16 == 0
    for tol, (rank, y) in res.items():
        assert relerr(y, y_ref) < TOL_MATVEC, (tol, rank)
    assert relerr(res[1e-6][1], res[-1.0][1]) < 1e-5


def test_mixed_precision_solve_and_energy(born):
    """Mixed-precision solve of the Born ion: same solution and energy as the oracle."""
    import paper_1710_06316_gb300 as pb
    mol, h0, o = born
    with pb.Handle.for_molecule(mol, order=6, precision=1) as h:
        f, hh, info = h.solve()
        E = h.energy()
    ref = o.solve(mol.atoms, mol.q)
    assert info["status"] == "OK"
    assert relerr(np.concatenate([f, hh]), np.concatenate([ref["f"], ref["h"]])) < 1e-4
    assert abs(E / ref["energy"] - 1) < 1e-4


@pytest.fixture(scope="module")
def small_globule():
    # ~23.6k nodes; the raw isosurface (t_clip 0.01, no smoothing) keeps its sliver
    # triangles, a stress case for the near-field quadrature
    mol = synthetic.globule(n_atoms=200, t_clip=0.01, smooth=0)
    o = oracle.Oracle.for_molecule(mol)
    x = synthetic.random_unknowns(mol.n_nodes, 21)
    return mol, o, x, o.matvec(x)


@pytest.mark.parametrize("precision", [0, 1])
def test_globule_matvec_adaptive_tree(small_globule, precision):
    """Synthetic globular molecule (compact walk + Gaussian isosurface): a non-uniform
    adaptive tree with lists 3 and 4 in play; full product against the oracle."""
    import paper_1710_06316_gb300 as pb
    mol, o, x, y_ref = small_globule
    with pb.Handle.for_molecule(mol, order=6, leaf_cap=64, precision=precision) as h:
        inf = h.info()
        assert inf["n_list_w"] > 0 and inf["n_list_x"] > 0 and inf["n_levels"] >= 5
        if precision == 0:
            check_tree_coverage(h)
        y = gpu_matvec(h, x)
    n = mol.n_nodes
    assert relerr(y, y_ref) < TOL_MATVEC
    assert relerr(y[:n], y_ref[:n]) < TOL_MATVEC
    assert relerr(y[n:], y_ref[n:]) < TOL_MATVEC


def test_globule_solve_and_energy():
    import paper_1710_06316_gb300 as pb
    mol = synthetic.globule(n_atoms=40, index=12)
    o = oracle.Oracle.for_molecule(mol)
    ref = o.solve(mol.atoms, mol.q)
    with pb.Handle.for_molecule(mol, order=6, leaf_cap=64, precision=1) as h:
        f, hh, info = h.solve()
        E = h.energy()
    assert info["status"] == "OK"
    assert relerr(np.concatenate([f, hh]), np.concatenate([ref["f"], ref["h"]])) < 1e-4
    assert abs(E / ref["energy"] - 1) < 1e-4


@pytest.mark.parametrize("precision", [0, 1])
def test_paper_sphere_energy(precision):
    """The paper's spherical case (Sec. 5): R = 50 A, +50 e at the centre, 0 mM salt,
    655,362 nodes / 1,310,720 triangles.  The paper's analytic energy is -4046 kcal/mol and
    its 3- and 6-digit runs were 0.47% and 0.29% off; the solve here must land within the
    paper's own error band, and within 0.1% of the Born closed form (eps 2/80)."""
    import os
    import paper_1710_06316_gb300 as pb
    g = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "paper_sphere.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            g[k] = float(v)
    mol = synthetic.paper_sphere()
    assert mol.n_nodes == int(g["n_nodes"]) and mol.n_tris == int(g["n_triangles"])
    with pb.Handle.for_molecule(mol, order=6, tol=1e-6, precision=precision) as h:
        f, hh, info = h.solve()
        E = h.energy()
    assert info["status"] == "OK"
    e_paper = g["analytic_energy_kcal_mol"]
    assert abs(E / e_paper - 1) < g["afmpb_6digit_rel_error"]
    assert abs(E / born_energy(50.0, 50.0, 2.0, 80.0, 0.0) - 1) < 1e-3


def test_tiny_mesh_without_far_field():
    """Icosahedron (12 nodes): one leaf, no multipole levels; all pairs by P2P."""
    import paper_1710_06316_gb300 as pb
    xyz, tri = synthetic.icosphere(0, radius=1.5)
    o = oracle.Oracle(xyz, tri, 2.0, 80.0, 0.3)
    x = synthetic.random_unknowns(12, 1)
    with pb.Handle(xyz, tri, eps_in=2.0, eps_out=80.0, kappa=0.3) as h:
        assert h.info()["n_m2l_pairs"] == 0
        y = gpu_matvec(h, x)
    assert relerr(y, o.matvec(x)) < 1e-5


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("xkind", ["smooth", "random"])
def test_kirkwood_full_size_sampled_rows(precision, xkind):
    """Kirkwood sphere at full size (163,842 nodes); precision 1 with its default leaf
    capacity is the bench's launch configuration.  4,096 rows sampled and computed one by
    one by the oracle, for a smooth x and for a random one (every near-field and P2P
    coefficient then counts with its own sign)."""
    import paper_1710_06316_gb300 as pb
    mol = synthetic.kirkwood_sphere()
    o = oracle.Oracle.for_molecule(mol)
    x = synthetic.smooth_unknowns(mol.xyz, 1) if xkind == "smooth" else synthetic.random_unknowns(mol.n_nodes, 13)
    with pb.Handle.for_molecule(mol, order=6, precision=precision) as h:
        y = gpu_matvec(h, x)
    rng = np.random.default_rng(7)
    rows = np.sort(rng.choice(mol.n_nodes, 4096, replace=False))
    y1, y2 = o.matvec_rows(rows, x)
    n = mol.n_nodes
    got = np.concatenate([y[rows], y[n + rows]])
    ref = np.concatenate([y1, y2])
    assert relerr(got, ref) < TOL_MATVEC


def test_bounded_wait_expires_and_the_context_stays_usable():
    """Failure path of the device waits, triggered on purpose: a wait on an mbarrier that
    nothing arrives at gives up after its poll limit and reports it; a product on the same
    context afterwards still matches the oracle."""
    import paper_1710_06316_gb300 as pb
    assert pb.selftest_bounded_wait(2000) is True
    mol = synthetic.born_ion(subdiv=3)
    x = synthetic.random_unknowns(mol.n_nodes, 4)
    with pb.Handle.for_molecule(mol, order=6, precision=1) as h:
        y = gpu_matvec(h, x)
    assert relerr(y, oracle.Oracle.for_molecule(mol).matvec(x)) < TOL_MATVEC


@pytest.mark.parametrize("subdiv,precision", [(5, 0), (5, 1)])
def test_folded_product_equals_its_parts(subdiv, precision):
    """The whole product folds the near-field correction into the P2P sums on the P2P
    branch (Eq. 5 assembled after the join); the part products keep the serialised
    combine.  Whole = diagonal + far + near to FP32 rounding of the reordered sums, on
    each block, with a random x; and both against the oracle at the product bar."""
    import paper_1710_06316_gb300 as pb
    mol = synthetic.kirkwood_sphere(subdiv=subdiv, kappa=0.2)
    rng = np.random.default_rng(31)
    x = rng.standard_normal(2 * mol.n_nodes)
    with pb.Handle.for_molecule(mol, order=6, precision=precision) as h:
        y = gpu_matvec(h, x, pb.PART_ALL)
        parts = sum(gpu_matvec(h, x, p) for p in (pb.PART_DIAG, pb.PART_FAR, pb.PART_NEAR))
    n = mol.n_nodes
    for blk in (slice(0, n), slice(n, 2 * n)):
        assert relerr(y[blk], parts[blk]) < 2e-6
    ref = oracle.Oracle.for_molecule(mol).matvec(x)
    for blk in (slice(0, n), slice(n, 2 * n)):
        assert relerr(y[blk], ref[blk]) < TOL_MATVEC
