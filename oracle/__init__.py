"""FP64 CPU oracle for the node-patch PB matvec (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The product library never links or calls it.  The C source
(``afmpb_oracle.c``) is compiled with gcc into ``liborc.so`` beside it.

Every routine follows the paper's equations (Sec. 2 Eq. 3-6 for the operator, Eq. 7 and
Sec. 3.4 for GMRES); see the header of ``afmpb_oracle.c`` for the readings taken where
the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "afmpb_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lib = None

K_C = 332.0636  # kcal A / (mol e^2); reading R7


def compile_source(src: str, out: str) -> str:
    """gcc (-O2, OpenMP, portable flags only) of one oracle source into a shared library."""
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           src, "-o", out, "-lm"])
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into ``liborc.so`` beside its source when the source is newer."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        compile_source(_SRC, tmp)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = configure(C.CDLL(_LIB))
    return _lib


def configure(lib):
    """Declare the argument and return types of the oracle's entry points on a loaded
    copy of the library (the tests also load copies compiled from altered sources)."""
    P = C.c_void_p
    i64, dbl, i32 = C.c_int64, C.c_double, C.c_int
    lib.orc_create.restype = P
    lib.orc_create.argtypes = [i64, P, i64, P, P, dbl, dbl, dbl, dbl]
    lib.orc_destroy.argtypes = [P]
    lib.orc_set_quadrature.argtypes = [P, i32, dbl, i32]
    lib.orc_get_geometry.argtypes = [P, P, P, P]
    lib.orc_alpha.restype = dbl
    lib.orc_alpha.argtypes = [P]
    lib.orc_mesh_check.restype = i32
    lib.orc_mesh_check.argtypes = [i64, i64, P, P, P, P]
    lib.orc_coeffs.argtypes = [P, i64, P, P, i32, P]
    lib.orc_tri_quad.argtypes = [P, P, P, P, P, P, P, P]
    lib.orc_surface_quad.argtypes = [P, i64, P, P, P]
    lib.orc_kernel_eval.argtypes = [dbl, i64, P, P, P, P, P]
    lib.orc_is_near.restype = i32
    lib.orc_is_near.argtypes = [P, i64, i64]
    lib.orc_build_near.restype = i64
    lib.orc_build_near.argtypes = [P]
    lib.orc_get_near.argtypes = [P, P, P, P]
    lib.orc_matvec.argtypes = [P, P, P, i32]
    lib.orc_matvec_rows.argtypes = [P, i64, P, P, P, i32]
    lib.orc_assemble.argtypes = [P, P]
    lib.orc_rhs.argtypes = [P, i64, P, P, P]
    lib.orc_rhs_rows.argtypes = [P, i64, P, P, i64, P, P]
    lib.orc_energy.restype = dbl
    lib.orc_energy.argtypes = [P, i64, P, P, P, P, P]
    lib.orc_gmres.restype = i32
    lib.orc_gmres.argtypes = [P, P, P, P, i32, i32, dbl, dbl, dbl, P]
    lib.orc_num_threads.restype = i32
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def mesh_check(xyz, tri):
    """Returns (code, euler, signed_volume); code 0 = closed, manifold, outward."""
    lib = _load()
    xyz = _f64(xyz)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    e = np.zeros(1, np.int64)
    v = np.zeros(1, np.float64)
    code = lib.orc_mesh_check(xyz.shape[0], tri.shape[0], _p(tri), _p(xyz), _p(e), _p(v))
    return int(code), int(e[0]), float(v[0])


def kernel_eval(kappa, x, n0, y, n):
    """Eight kernel values per pair: G, dG/dn, dG/dn0, d2G/dn0dn, u, du/dn, du/dn0,
    d2u/dn0dn  (n = source normal at y, n0 = target normal at x)."""
    lib = _load()
    x, n0, y, n = (_f64(np.atleast_2d(a)) for a in (x, n0, y, n))
    out = np.zeros((x.shape[0], 8))
    lib.orc_kernel_eval(float(kappa), x.shape[0], _p(x), _p(n0), _p(y), _p(n), _p(out))
    return out


class Oracle:
    """One mesh + physical parameters.  All results are FP64 numpy arrays in the
    caller's node order; x = [f; h] and y = [y1; y2] have length 2N."""

    FAR, NEAR, AUTO = 0, 1, 2

    def __init__(self, xyz, tri, eps_in, eps_out, kappa, c_near=2.0, normals=None):
        self._lib = _load()
        self.xyz = _f64(xyz)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.n = self.xyz.shape[0]
        self.eps_in, self.eps_out, self.kappa = float(eps_in), float(eps_out), float(kappa)
        nrm = None if normals is None else _f64(normals)
        self._nrm_keep = nrm
        self._h = self._lib.orc_create(self.n, _p(self.xyz), self.tri.shape[0], _p(self.tri),
                                       None if nrm is None else _p(nrm), self.eps_in,
                                       self.eps_out, self.kappa, float(c_near))
        self.alpha = self._lib.orc_alpha(self._h)
        self.ebar = self.eps_out / self.eps_in

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    @classmethod
    def for_molecule(cls, mol, **kw):
        return cls(mol.xyz, mol.tri, mol.eps_in, mol.eps_out, mol.kappa, **kw)

    def set_quadrature(self, max_depth=6, refine_ratio=3.0, gl_n=16):
        self._lib.orc_set_quadrature(self._h, int(max_depth), float(refine_ratio), int(gl_n))

    def geometry(self):
        a = np.zeros(self.n)
        nrm = np.zeros((self.n, 3))
        rho = np.zeros(self.n)
        self._lib.orc_get_geometry(self._h, _p(a), _p(nrm), _p(rho))
        return a, nrm, rho

    def coeffs(self, p, t, rule=AUTO):
        p = np.ascontiguousarray(p, dtype=np.int64).ravel()
        t = np.ascontiguousarray(t, dtype=np.int64).ravel()
        out = np.zeros((p.size, 4))
        self._lib.orc_coeffs(self._h, p.size, _p(p), _p(t), int(rule), _p(out))
        return out

    def tri_quad(self, x, n0, a, b, c, ns):
        out = np.zeros(4)
        arrs = [_f64(v) for v in (x, n0, a, b, c, ns)]
        self._lib.orc_tri_quad(self._h, *[_p(v) for v in arrs], _p(out))
        return out

    def surface_quad(self, x, n0):
        x = _f64(np.atleast_2d(x))
        n0 = _f64(np.atleast_2d(n0))
        out = np.zeros((x.shape[0], 4))
        self._lib.orc_surface_quad(self._h, x.shape[0], _p(x), _p(n0), _p(out))
        return out

    def is_near(self, p, t):
        return bool(self._lib.orc_is_near(self._h, int(p), int(t)))

    def near_csr(self):
        nnz = self._lib.orc_build_near(self._h)
        rp = np.zeros(self.n + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        coef = np.zeros((nnz, 4))
        self._lib.orc_get_near(self._h, _p(rp), _p(col), _p(coef))
        return rp, col, coef

    def matvec(self, x, mode=0):
        """mode 0: the operator of Eq. 5; mode 1: alpha x + far rule for all t != p."""
        x = _f64(x)
        y = np.zeros(2 * self.n)
        self._lib.orc_matvec(self._h, _p(x), _p(y), int(mode))
        return y

    def matvec_rows(self, rows, x, mode=0):
        """Rows of y: returns (y1[rows], y2[rows])."""
        rows = np.ascontiguousarray(rows, dtype=np.int64).ravel()
        x = _f64(x)
        y = np.zeros(2 * rows.size)
        self._lib.orc_matvec_rows(self._h, rows.size, _p(rows), _p(x), _p(y), int(mode))
        return y[0::2].copy(), y[1::2].copy()

    def assemble(self):
        M = np.zeros((2 * self.n, 2 * self.n))
        self._lib.orc_assemble(self._h, _p(M))
        return M

    def rhs(self, atoms, q):
        atoms = _f64(np.atleast_2d(atoms))
        q = _f64(q)
        b = np.zeros(2 * self.n)
        self._lib.orc_rhs(self._h, q.size, _p(atoms), _p(q), _p(b))
        return b

    def rhs_rows(self, rows, atoms, q):
        """Rows of b: returns (b1[rows], b2[rows])."""
        atoms = _f64(np.atleast_2d(atoms))
        q = _f64(q)
        rows = np.ascontiguousarray(rows, dtype=np.int64).ravel()
        b = np.zeros(2 * rows.size)
        self._lib.orc_rhs_rows(self._h, q.size, _p(atoms), _p(q), rows.size, _p(rows), _p(b))
        return b[0::2].copy(), b[1::2].copy()

    def energy(self, atoms, q, f, h, return_phi=False):
        atoms = _f64(np.atleast_2d(atoms))
        q, f, h = _f64(q), _f64(f), _f64(h)
        phi = np.zeros(q.size)
        E = self._lib.orc_energy(self._h, q.size, _p(atoms), _p(q), _p(f), _p(h), _p(phi))
        return (E, phi) if return_phi else E

    def gmres(self, b, restart=80, max_restart=5, rel_tol=1e-6, abs_tol=0.0, dense=None,
              eta=1e-3):
        """Restarted GMRES; ``dense`` = an assembled matrix to use for the products (or
        None for the matrix-free operator).  Returns (x, info dict, converged)."""
        b = _f64(b)
        x = np.zeros(2 * self.n)
        info = np.zeros(5)
        M = None if dense is None else np.ascontiguousarray(dense, dtype=np.float64)
        rc = self._lib.orc_gmres(self._h, None if M is None else _p(M), _p(b), _p(x),
                                 int(restart), int(max_restart), float(rel_tol),
                                 float(abs_tol), float(eta), _p(info))
        d = dict(iters=int(info[0]), inner=int(info[1]), restarts=int(info[2]),
                 res_est=float(info[3]), res_true=float(info[4]))
        return x, d, rc == 0

    def solve(self, atoms, q, rel_tol=1e-6, restart=80, max_restart=5):
        """RHS -> GMRES -> energy, the paper's solution flow (Sec. 2 list)."""
        b = self.rhs(atoms, q)
        x, info, ok = self.gmres(b, restart=restart, max_restart=max_restart, rel_tol=rel_tol)
        f, h = x[: self.n], x[self.n:]
        E = self.energy(atoms, q, f, h)
        return dict(f=f, h=h, energy=E, info=info, converged=ok, b=b)
