"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only *generates inputs* -- meshes, atom positions and charges.  It holds
none of the method's arithmetic (no patch geometry, kernels, quadrature, matvec, GMRES
or energy); both the FP64 oracle and the CUDA library receive exactly what these
functions return.

Workloads (all seeded with ``SEED_BASE + index`` through numpy's PCG64):

* ``born_ion``        -- sphere radius 2 A, +1 e at the centre, icosphere subdivision 4
                          (2,562 nodes / 5,120 triangles).  Stands in for the paper's
                          spherical validation case (Sec. 5) at small size.
* ``kirkwood_sphere`` -- sphere radius 20 A, 64 charges uniform in r < 16 A with
                          q ~ U(-1, 1), icosphere subdivision 7 (163,842 nodes).
* ``paper_sphere``    -- the paper's Sec. 5 sphere: R = 50 A, +50 e at the centre,
                          icosphere subdivision 8 (655,362 nodes, 1,310,720 triangles).
* ``globule``         -- a compact self-avoiding random walk of atoms with a
                          summed-Gaussian molecular surface (see ``globule``).

Triangles are returned counter-clockwise when seen from the solvent (outward normals),
which is the orientation the library's C-ABI requires.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 1710063160


@dataclass
class Molecule:
    """A synthetic molecule: surface mesh plus point charges (Angstrom, e)."""

    name: str
    xyz: np.ndarray      # [n_nodes, 3] float64
    tri: np.ndarray      # [n_tris, 3] int32, CCW seen from outside
    atoms: np.ndarray    # [n_atoms, 3] float64
    q: np.ndarray        # [n_atoms] float64
    eps_in: float
    eps_out: float
    kappa: float
    meta: dict

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tri.shape[0])


def rng_for(index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index))


# ----------------------------------------------------------------------------------
# icosphere
# ----------------------------------------------------------------------------------
def _icosahedron():
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([
        [-1, g, 0], [1, g, 0], [-1, -g, 0], [1, -g, 0],
        [0, -1, g], [0, 1, g], [0, -1, -g], [0, 1, -g],
        [g, 0, -1], [g, 0, 1], [-g, 0, -1], [-g, 0, 1],
    ], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    # make every face counter-clockwise seen from outside
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    s = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c)
    f[s < 0] = f[s < 0][:, [0, 2, 1]]
    return v, f


def icosphere(subdiv: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Unit icosahedron refined ``subdiv`` times (1 -> 4 split, midpoints pushed to the
    sphere), scaled by ``radius``.  Nodes: 10 * 4**subdiv + 2."""
    v, f = _icosahedron()
    for _ in range(subdiv):
        nv = v.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e.sort(axis=1)
        key = e[:, 0] * (nv + 1) + e[:, 1]
        uniq, inv = np.unique(key, return_inverse=True)
        ea = uniq // (nv + 1)
        eb = uniq % (nv + 1)
        mid = v[ea] + v[eb]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid], axis=0)
        nt = f.shape[0]
        mab = nv + inv[0:nt]
        mbc = nv + inv[nt:2 * nt]
        mca = nv + inv[2 * nt:3 * nt]
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        f = np.concatenate([
            np.stack([a, mab, mca], 1),
            np.stack([mab, b, mbc], 1),
            np.stack([mca, mbc, c], 1),
            np.stack([mab, mbc, mca], 1),
        ], axis=0)
    xyz = v * float(radius) + np.asarray(center, dtype=np.float64)[None, :]
    return xyz.astype(np.float64), f.astype(np.int32)


# ----------------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------------
def born_ion(subdiv: int = 4, radius: float = 2.0, q: float = 1.0, eps_in: float = 1.0,
             eps_out: float = 80.0, kappa: float = 0.104) -> Molecule:
    xyz, tri = icosphere(subdiv, radius)
    return Molecule("born_ion", xyz, tri, np.zeros((1, 3)), np.array([float(q)]),
                    eps_in, eps_out, kappa, {"radius": radius, "subdiv": subdiv})


def paper_sphere(subdiv: int = 8) -> Molecule:
    """The paper's spherical test (Sec. 5): R = 50 A, +50 e at the centre, 0 mM salt;
    subdivision 8 gives its 655,362 nodes / 1,310,720 triangles."""
    m = born_ion(subdiv=subdiv, radius=50.0, q=50.0, eps_in=2.0, eps_out=80.0, kappa=0.0)
    m.name = "paper_sphere"
    return m


def uniform_ball_charges(rng: np.random.Generator, n: int, r_max: float):
    r = r_max * rng.random(n) ** (1.0 / 3.0)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * r[:, None]


def kirkwood_sphere(subdiv: int = 7, radius: float = 20.0, n_charges: int = 64,
                    r_charges: float = 16.0, eps_in: float = 2.0, eps_out: float = 80.0,
                    kappa: float = 0.104, index: int = 1) -> Molecule:
    rng = rng_for(index)
    atoms = uniform_ball_charges(rng, n_charges, r_charges)
    q = rng.uniform(-1.0, 1.0, n_charges)
    xyz, tri = icosphere(subdiv, radius)
    return Molecule("kirkwood_sphere", xyz, tri, atoms, q, eps_in, eps_out, kappa,
                    {"radius": radius, "subdiv": subdiv})


# ----------------------------------------------------------------------------------
# synthetic globular molecule: compact self-avoiding walk + Gaussian isosurface
# ----------------------------------------------------------------------------------
def compact_walk(rng: np.random.Generator, n_atoms: int, step: float = 1.5, min_dist: float = 1.0,
                 r_confine: float | None = None, max_reject: int = 50, axes=None):
    """Self-avoiding random walk of n_atoms points: isotropic steps of `step`, a step is
    rejected if it comes within `min_dist` of an earlier point or leaves the confinement
    region; after `max_reject` rejections in a row the walk backtracks one point.
    The region is the ellipsoid with semi-axes `axes` when given, else a sphere; the
    default radius 38.7 (N/20000)^(1/3) A gives a protein-like density."""
    if r_confine is None:
        r_confine = 38.7 * (n_atoms / 20000.0) ** (1.0 / 3.0)
    inv_ax = None if axes is None else 1.0 / np.asarray(axes, dtype=np.float64)
    cell = min_dist
    grid: dict = {}
    pts = [np.zeros(3)]

    def key(p):
        return (int(np.floor(p[0] / cell)), int(np.floor(p[1] / cell)), int(np.floor(p[2] / cell)))

    grid.setdefault(key(pts[0]), []).append(0)
    fails = 0
    while len(pts) < n_atoms:
        d = rng.standard_normal(3)
        c = pts[-1] + step * d / np.linalg.norm(d)
        if inv_ax is None:
            ok = np.dot(c, c) <= r_confine * r_confine
        else:
            u = c * inv_ax
            ok = np.dot(u, u) <= 1.0
        if ok:
            kx, ky, kz = key(c)
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for j in grid.get((kx + dx, ky + dy, kz + dz), ()):
                            if np.sum((pts[j] - c) ** 2) < min_dist * min_dist:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
        if ok:
            grid.setdefault(key(c), []).append(len(pts))
            pts.append(c)
            fails = 0
        else:
            fails += 1
            if fails >= max_reject and len(pts) > 1:
                last = pts.pop()
                grid[key(last)].remove(len(pts))
                fails = 0
    return np.array(pts)


def gaussian_density(atoms, radii, origin, h, shape, beta=2.3, cutoff=1e-4):
    """rho(x) = sum_i exp(beta (1 - |x - x_i|^2 / r_i^2)) on a regular grid."""
    rho = np.zeros(shape)
    for a, r in zip(atoms, radii):
        reach = r * np.sqrt(1.0 - np.log(cutoff) / beta)
        lo = np.maximum(np.floor((a - reach - origin) / h).astype(int), 0)
        hi = np.minimum(np.ceil((a + reach - origin) / h).astype(int) + 1, np.array(shape))
        xs = [origin[d] + h * np.arange(lo[d], hi[d]) - a[d] for d in range(3)]
        d2 = xs[0][:, None, None] ** 2 + xs[1][None, :, None] ** 2 + xs[2][None, None, :] ** 2
        rho[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] += np.exp(beta * (1.0 - d2 / (r * r)))
    return rho


# Kuhn split of the unit cube into 6 tetrahedra along the (0 -> 7) diagonal; corner c has
# offset (c & 1, (c >> 1) & 1, (c >> 2) & 1).  The split is the same in every cube, so
# neighbouring tetrahedra share faces and the extracted surface is closed.
_KUHN = np.array([[0, 1, 3, 7], [0, 1, 5, 7], [0, 2, 3, 7], [0, 2, 6, 7], [0, 4, 5, 7], [0, 4, 6, 7]])


def isosurface(values, origin, h, level=1.0, t_clip=0.01):
    """Marching tetrahedra on a regular grid: the closed surface {values = level} with
    triangles counter-clockwise seen from the low side (outward when the inside has
    values > level).  Vertices lie on grid edges and are shared by edge."""
    v = np.array(values, dtype=np.float64) - level
    v[np.abs(v) < 1e-9] = 1e-9
    nx, ny, nz = v.shape
    inside = v > 0
    # cubes with mixed signs
    corners = np.stack([inside[(c & 1):nx - 1 + (c & 1), ((c >> 1) & 1):ny - 1 + ((c >> 1) & 1),
                               ((c >> 2) & 1):nz - 1 + ((c >> 2) & 1)] for c in range(8)], axis=-1)
    mixed = corners.any(-1) & ~corners.all(-1)
    ci, cj, ck = np.nonzero(mixed)
    off = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)])
    tris, keys_all, tpos = [], [], []
    for tet in _KUHN:
        gi = ci[:, None] + off[tet][:, 0][None, :]
        gj = cj[:, None] + off[tet][:, 1][None, :]
        gk = ck[:, None] + off[tet][:, 2][None, :]
        gid = (gi * ny + gj) * nz + gk                        # [m, 4] global grid ids
        val = v[gi, gj, gk]
        ins = val > 0
        cnt = ins.sum(1)
        pos = origin[None, None, :] + h * np.stack([gi, gj, gk], -1)
        for m_in in (1, 2, 3):
            sel = np.nonzero(cnt == m_in)[0]
            if sel.size == 0:
                continue
            order = np.argsort(~ins[sel], axis=1, kind="stable")   # inside vertices first
            ids = np.take_along_axis(gid[sel], order, 1)
            vals = np.take_along_axis(val[sel], order, 1)
            ps = np.take_along_axis(pos[sel], order[:, :, None], 1)
            if m_in == 1:
                cuts = [[(0, 1), (0, 2), (0, 3)]]
            elif m_in == 3:
                cuts = [[(0, 3), (1, 3), (2, 3)]]
            else:
                cuts = [[(0, 2), (0, 3), (1, 3)], [(0, 2), (1, 3), (1, 2)]]
            cin = ps[:, :m_in].mean(1)
            cout = ps[:, m_in:].mean(1)
            for tri_cut in cuts:
                vp, vk = [], []
                for a, b in tri_cut:
                    t = np.clip(vals[:, a] / (vals[:, a] - vals[:, b]), t_clip, 1.0 - t_clip)
                    vp.append(ps[:, a] + t[:, None] * (ps[:, b] - ps[:, a]))
                    lo_id = np.minimum(ids[:, a], ids[:, b])
                    hi_id = np.maximum(ids[:, a], ids[:, b])
                    vk.append(lo_id * (nx * ny * nz) + hi_id)
                vp = np.stack(vp, 1)
                vk = np.stack(vk, 1)
                nrm = np.cross(vp[:, 1] - vp[:, 0], vp[:, 2] - vp[:, 0])
                flip = np.einsum("ij,ij->i", nrm, cout - cin) < 0
                vk[flip] = vk[flip][:, [0, 2, 1]]
                vp[flip] = vp[flip][:, [0, 2, 1]]
                keys_all.append(vk)
                tpos.append(vp)
    keys = np.concatenate(keys_all)
    vps = np.concatenate(tpos)
    uniq, first, inv = np.unique(keys.ravel(), return_index=True, return_inverse=True)
    xyz = vps.reshape(-1, 3)[first]
    tri = inv.reshape(-1, 3)
    return xyz, tri


def taubin_smooth(xyz, tri, iters: int = 10, lam: float = 0.5, mu: float = -0.53):
    """Taubin's lambda/mu smoothing (SIGGRAPH 1995): alternating umbrella steps
    x += lam (mean of neighbours - x) and x += mu (...), which evens out the triangle
    shapes of an isosurface without the shrinkage of plain Laplacian smoothing.  The
    connectivity is unchanged."""
    from scipy.sparse import coo_matrix, diags
    n = xyz.shape[0]
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    e = np.concatenate([e, e[:, ::-1]])
    A = coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n)).tocsr()
    A.data[:] = 1.0
    W = diags(1.0 / np.asarray(A.sum(1)).ravel()) @ A
    x = np.array(xyz, dtype=np.float64)
    for _ in range(iters):
        x = x + lam * (W @ x - x)
        x = x + mu * (W @ x - x)
    return x


def outer_component(xyz, tri):
    """Keep the connected surface component that contains the vertex of largest x."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    n = xyz.shape[0]
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    g = coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
    _, lab = connected_components(g, directed=False)
    keep = lab == lab[np.argmax(xyz[:, 0])]
    tri = tri[keep[tri[:, 0]]]
    used = np.unique(tri.ravel())
    remap = -np.ones(n, dtype=np.int64)
    remap[used] = np.arange(used.size)
    return xyz[used], remap[tri].astype(np.int32)


def globule(n_atoms: int = 20000, index: int = 2, grid: float = 0.4, beta: float = 2.3,
            eps_in: float = 2.0, eps_out: float = 80.0, kappa: float = 0.104,
            r_confine: float | None = None, t_clip: float = 0.2, smooth: int = 10) -> Molecule:
    """Synthetic globular protein: compact self-avoiding walk (1.5 A steps, 1.0 A exclusion,
    confinement radius 38.7 (N/20000)^(1/3) A), atomic radii U(1.2, 2.0) A, partial charges
    N(0, 0.35) e shifted to zero net charge, molecular surface = outer component of the
    rho = 1 isosurface of the summed-Gaussian density on a `grid`-A lattice, with edge
    parameters clipped to [t_clip, 1 - t_clip] and `smooth` Taubin smoothing passes.
    t_clip = 0.01 and smooth = 0 keep the raw isosurface, whose sliver triangles slow
    GMRES down by an order of magnitude on large meshes."""
    rng = rng_for(index)
    atoms = compact_walk(rng, n_atoms, r_confine=r_confine)
    radii = rng.uniform(1.2, 2.0, n_atoms)
    q = rng.normal(0.0, 0.35, n_atoms)
    q -= q.mean()
    pad = 2.5 * radii.max() + 2 * grid
    lo = atoms.min(0) - pad
    hi = atoms.max(0) + pad
    shape = tuple(int(np.ceil((hi[d] - lo[d]) / grid)) + 1 for d in range(3))
    rho = gaussian_density(atoms, radii, lo, grid, shape, beta=beta)
    xyz, tri = isosurface(rho, lo, grid, level=1.0, t_clip=t_clip)
    xyz, tri = outer_component(xyz, tri)
    if smooth > 0:
        xyz = taubin_smooth(xyz, tri, smooth)
    return Molecule("globule", xyz, tri, atoms, q, eps_in, eps_out, kappa,
                    {"n_atoms": n_atoms, "grid": grid, "beta": beta, "t_clip": t_clip, "smooth": smooth})


def icosahedral_rotations():
    """The 60 proper rotations of the icosahedron: the closure of a 72-degree turn about
    the vertex axis (0, 1, phi) and a 120-degree turn about the face axis (1, 1, 1)."""
    phi = 0.5 * (1.0 + np.sqrt(5.0))

    def turn(axis, ang):
        a = np.asarray(axis, dtype=np.float64)
        a = a / np.linalg.norm(a)
        K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
        return np.eye(3) + np.sin(ang) * K + (1.0 - np.cos(ang)) * K @ K

    gens = [turn((0.0, 1.0, phi), 2.0 * np.pi / 5.0), turn((1.0, 1.0, 1.0), 2.0 * np.pi / 3.0)]
    group = [np.eye(3)]
    frontier = [np.eye(3)]
    while frontier:
        nxt = []
        for g in frontier:
            for s in gens:
                m = s @ g
                if not any(np.abs(m - e).max() < 1e-9 for e in group):
                    group.append(m)
                    nxt.append(m)
        frontier = nxt
    return np.array(group)


def _spread_direction(rots, samples: int = 4000, seed: int = 7):
    """A unit vector whose 60 images under `rots` are as far apart as possible (best of a
    seeded random sample of directions)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((samples, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    imgs = np.einsum("gij,sj->sgi", rots, d)                    # [samples, 60, 3]
    best, best_v = None, -1.0
    for k in range(samples):
        p = imgs[k]
        g = p @ p.T
        np.fill_diagonal(g, -2.0)
        v = 1.0 - g.max()                                       # 1 - cos of the smallest angle
        if v > best_v:
            best, best_v = d[k], v
    return best


def capsid(n_atoms: int = 20000, copies: int = 60, r_shell: float = 250.0, thickness: float = 40.0,
           grid: float = 1.2, index: int = 4, beta: float = 2.3, eps_in: float = 2.0, eps_out: float = 80.0,
           kappa: float = 0.104, t_clip: float = 0.2, smooth: int = 10) -> Molecule:
    """Virus-capsid stand-in: `copies` (at most 60) copies of one globule placed by the
    icosahedral rotations on a shell of mean radius r_shell.  The globule is a compact walk
    confined to an oblate ellipsoid (radial semi-axis thickness/2 + 5 A, tangential semi-axes
    chosen for a protein-like density), radii U(1.2, 2.0) A, charges N(0, 0.35) e shifted to
    zero net; its surface is the outer component of the rho = 1 Gaussian isosurface on a
    `grid`-A lattice (edge parameters clipped to [t_clip, 1 - t_clip], `smooth` Taubin
    passes, as for the globule), and every copy carries the same mesh, moved rigidly.  The copies are
    checked to be disjoint (bounding spheres apart), so the surface is `copies` closed
    components."""
    rng = rng_for(index)
    a_r = 0.5 * thickness + 5.0
    vol = n_atoms * (4.0 / 3.0 * np.pi * 38.7 ** 3 / 20000.0)  # the globule's atom density
    a_t = np.sqrt(vol / (4.0 / 3.0 * np.pi * a_r))
    atoms = compact_walk(rng, n_atoms, axes=(a_t, a_t, a_r))
    radii = rng.uniform(1.2, 2.0, n_atoms)
    q = rng.normal(0.0, 0.35, n_atoms)
    q -= q.mean()
    pad = 2.5 * radii.max() + 2 * grid
    lo = atoms.min(0) - pad
    hi = atoms.max(0) + pad
    shape = tuple(int(np.ceil((hi[d] - lo[d]) / grid)) + 1 for d in range(3))
    rho = gaussian_density(atoms, radii, lo, grid, shape, beta=beta)
    xyz, tri = isosurface(rho, lo, grid, level=1.0, t_clip=t_clip)
    xyz, tri = outer_component(xyz, tri)
    if smooth > 0:
        xyz = taubin_smooth(xyz, tri, smooth)
    rots = icosahedral_rotations()[:copies]
    d = _spread_direction(icosahedral_rotations())
    # rotation taking the z axis to d (Rodrigues about z x d)
    z = np.array([0.0, 0.0, 1.0])
    v = np.cross(z, d)
    s_, c_ = np.linalg.norm(v), float(np.dot(z, d))
    K = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
    R0 = np.eye(3) + K + K @ K * ((1.0 - c_) / max(s_ * s_, 1e-300))
    shift = np.array([0.0, 0.0, r_shell])
    base_xyz = (xyz + shift) @ R0.T
    base_atoms = (atoms + shift) @ R0.T
    centre = R0 @ shift
    r_bound = np.linalg.norm(base_xyz - centre, axis=1).max()
    cs = np.einsum("gij,j->gi", rots, centre)
    dist = np.linalg.norm(cs[:, None, :] - cs[None, :, :], axis=2)
    np.fill_diagonal(dist, np.inf)
    if dist.min() <= 2.0 * r_bound:
        raise ValueError("capsid copies overlap: centre spacing %.1f A <= 2 x %.1f A"
                         % (dist.min(), r_bound))
    nb = xyz.shape[0]
    all_xyz = np.concatenate([base_xyz @ g.T for g in rots])
    all_tri = np.concatenate([tri + i * nb for i in range(len(rots))]).astype(np.int32)
    all_atoms = np.concatenate([base_atoms @ g.T for g in rots])
    all_q = np.tile(q, len(rots))
    return Molecule("capsid", all_xyz, all_tri, all_atoms, all_q, eps_in, eps_out, kappa,
                    {"n_atoms": n_atoms * len(rots), "copies": len(rots), "grid": grid,
                     "copy_nodes": nb, "r_shell": r_shell, "axes": (a_t, a_t, a_r)})


def random_unknowns(n_nodes: int, seed: int, dtype=np.float64):
    """A seeded test vector x = [f; h] of length 2N with O(1) entries."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 1000 + seed))
    return rng.uniform(-1.0, 1.0, 2 * n_nodes).astype(dtype)


def smooth_unknowns(xyz: np.ndarray, seed: int):
    """A smooth test vector (low-order harmonics of the node positions), the kind of
    field a converged solution looks like; avoids the white-noise worst case."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 2000 + seed))
    c = xyz - xyz.mean(axis=0)
    s = np.abs(c).max()
    c = c / s
    w = rng.standard_normal((2, 3))
    f = 1.0 + c @ w[0] + 0.5 * (c[:, 0] * c[:, 1])
    h = -0.5 + c @ w[1] + 0.3 * (c[:, 2] ** 2)
    return np.concatenate([f, h])
