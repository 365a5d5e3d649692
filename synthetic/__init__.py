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
