"""Python binding of libafmpb (GB300 node-patch Poisson-Boltzmann solver).

Argument marshalling only: every step of the product, the solve and the energy runs in
the CUDA library behind the C ABI of ``include/afmpb.h``.  Device buffers are passed as
raw pointers (``int``) or as objects with ``data_ptr()`` (PyTorch tensors); the binding
never computes anything itself and raises if the native library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

_lib = None

PART_DIAG, PART_FAR, PART_NEAR, PART_ALL = 1, 2, 4, 7
RESTART_NONE = -1
ORTH_CGS2, ORTH_ONE_REDUCTION = 0, 1
STATUS = {0: "OK", 1: "EINVAL", 2: "EMESH", 3: "ENOMEM", 4: "ECUDA", 5: "ENOCONV", 6: "ETIMEOUT",
          7: "EBUSY", 8: "ESTATE", 9: "EINTERNAL"}


class AfmpbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code
        self.status = STATUS.get(code, str(code))


class Mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tris", C.c_int64), ("xyz", C.c_void_p),
                ("tri", C.c_void_p), ("normals", C.c_void_p)]


class Charges(C.Structure):
    _fields_ = [("n", C.c_int64), ("xyz", C.c_void_p), ("q", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("leaf_cap", C.c_int), ("restart", C.c_int), ("max_restart", C.c_int),
                ("abs_tol", C.c_double), ("precision", C.c_int), ("near_c", C.c_double),
                ("stream", C.c_void_p), ("max_level", C.c_int), ("m2l_tol", C.c_double),
                ("charge_fmm", C.c_int), ("orth", C.c_int), ("m2l_method", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("res_est", C.c_double),
                ("res_true", C.c_double), ("bnorm", C.c_double), ("ms_setup", C.c_double),
                ("ms_matvec_total", C.c_double), ("ms_gmres", C.c_double),
                ("nnz_near", C.c_int64), ("n_boxes", C.c_int64), ("krylov_dim", C.c_int),
                ("second_passes", C.c_int)]


class Info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tris", C.c_int64), ("n_atoms", C.c_int64),
                ("n_boxes", C.c_int64), ("n_leaves", C.c_int64), ("n_levels", C.c_int64),
                ("nnz_near", C.c_int64), ("n_list_u", C.c_int64), ("n_list_v", C.c_int64),
                ("n_list_w", C.c_int64), ("n_list_x", C.c_int64), ("n_p2p_pairs", C.c_int64),
                ("n_m2l_pairs", C.c_int64), ("order", C.c_int), ("precision", C.c_int),
                ("device_bytes", C.c_int64), ("root_center", C.c_double * 3),
                ("root_half_width", C.c_double), ("ms_create", C.c_double * 6),
                ("m2l_rank", C.c_int), ("m2l_tables", C.c_int), ("device_bytes_peak", C.c_int64),
                ("leaf_cap", C.c_int), ("autotuned", C.c_int), ("charge_fmm", C.c_int),
                ("charge_fmm_boxes", C.c_int64)]


AUTOTUNE_MAX = 16
LEAF_CAP_AUTO = -1


class AutotuneReport(C.Structure):
    _fields_ = [("n_candidates", C.c_int), ("cap", C.c_int * AUTOTUNE_MAX),
                ("p2p_ms", C.c_double * AUTOTUNE_MAX), ("predicted_ms", C.c_double * AUTOTUNE_MAX),
                ("start_cap", C.c_int), ("best_cap", C.c_int), ("predicted_start_ms", C.c_double),
                ("predicted_best_ms", C.c_double), ("ms_per_m2l_pair", C.c_double),
                ("ms_per_box", C.c_double), ("ms_rest", C.c_double), ("ms_tuning", C.c_double),
                ("p2p_resident", C.c_int), ("p2p_units_per_block", C.c_int), ("m2l_runs_per_item", C.c_int),
                ("p2p_ms_default", C.c_double), ("p2p_ms_tuned", C.c_double),
                ("m2l_ms_default", C.c_double), ("m2l_ms_tuned", C.c_double)]


class Profile(C.Structure):
    _fields_ = [("n_stages", C.c_int), ("name", (C.c_char * 16) * 16), ("ms", C.c_double * 16),
                ("launches", C.c_int * 16), ("ms_graph", C.c_double), ("kernels_per_product", C.c_int)]


class Request(C.Structure):
    _fields_ = [("mesh", Mesh), ("charges", Charges), ("eps_in", C.c_double), ("eps_out", C.c_double),
                ("kappa", C.c_double), ("fmm_order", C.c_int), ("tol", C.c_double), ("options", Options),
                ("f_out", C.c_void_p), ("h_out", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("error", C.c_char * 160), ("energy_kcal_mol", C.c_double),
                ("info", SolveInfo), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("bytes_reserved", C.c_int64), ("bytes_used", C.c_int64),
                ("slot", C.c_int)]


class ServerInfo(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("running", C.c_int64), ("queued", C.c_int64), ("bytes_in_use", C.c_int64),
                ("bytes_high_water", C.c_int64), ("bytes_budget", C.c_int64),
                ("max_running", C.c_int64), ("slots", C.c_int), ("max_batch", C.c_int),
                ("batches", C.c_int64), ("batched_requests", C.c_int64)]


class PlanInput(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_boxes", C.c_int64), ("box_range", C.c_void_p),
                ("box_parent", C.c_void_p), ("u_ptr", C.c_void_p), ("u_idx", C.c_void_p),
                ("v_ptr", C.c_void_p), ("v_idx", C.c_void_p), ("w_ptr", C.c_void_p), ("w_idx", C.c_void_p),
                ("x_ptr", C.c_void_p), ("x_idx", C.c_void_p), ("near_ptr", C.c_void_p), ("near_col", C.c_void_p)]


class PlanRank(C.Structure):
    _fields_ = [("node_begin", C.c_int64), ("node_end", C.c_int64), ("n_halo", C.c_int64),
                ("n_send", C.c_int64), ("n_import_boxes", C.c_int64), ("n_shared_boxes", C.c_int64),
                ("work", C.c_double)]


def _struct_dict(s):
    out = {}
    for name, _ in s._fields_:
        v = getattr(s, name)
        out[name] = list(v) if hasattr(v, "__len__") else v
    return out


EXPORTS = ["afmpb_create", "afmpb_matvec", "afmpb_matvec_parts", "afmpb_matvec_host", "afmpb_solve",
           "afmpb_energy", "afmpb_rhs", "afmpb_get_geometry", "afmpb_get_near", "afmpb_get_tree",
           "afmpb_get_info", "afmpb_destroy", "afmpb_last_error", "afmpb_estimate_bytes",
           "afmpb_version", "afmpb_profile_product", "afmpb_energy_noalloc",
           "afmpb_server_create", "afmpb_server_submit", "afmpb_server_poll", "afmpb_server_wait",
           "afmpb_server_get_info", "afmpb_server_destroy", "afmpb_get_autotune",
           "afmpb_selftest_bounded_wait", "afmpb_sync", "afmpb_inject_wait_expiry",
           "afmpb_plan_create", "afmpb_plan_get_rank", "afmpb_plan_get_halo", "afmpb_plan_get_send",
           "afmpb_plan_get_boxes", "afmpb_plan_destroy", "afmpb_solve_batch",
           "afmpb_server_create_batched"]


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load libafmpb.so (building it with nvcc if needed).  Raises if it cannot load."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libafmpb.so is missing; run paper_1710_06316_gb300._build.build()")
    lib = C.CDLL(_build.LIB)
    P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int, C.c_double
    lib.afmpb_create.restype = I32
    lib.afmpb_create.argtypes = [C.POINTER(Mesh), C.POINTER(Charges), D, D, D, I32, D,
                                 C.POINTER(Options), C.POINTER(P)]
    for name in ("afmpb_matvec", "afmpb_matvec_host"):
        getattr(lib, name).restype = I32
        getattr(lib, name).argtypes = [P, P, P]
    for name in ("afmpb_sync", "afmpb_inject_wait_expiry"):
        getattr(lib, name).restype = I32
        getattr(lib, name).argtypes = [P]
    lib.afmpb_plan_create.restype = I32
    lib.afmpb_plan_create.argtypes = [C.POINTER(PlanInput), I32, C.POINTER(P)]
    lib.afmpb_plan_get_rank.restype = I32
    lib.afmpb_plan_get_rank.argtypes = [P, I32, C.POINTER(PlanRank)]
    for name in ("afmpb_plan_get_halo", "afmpb_plan_get_send"):
        getattr(lib, name).restype = I32
        getattr(lib, name).argtypes = [P, I32, P, P]
    lib.afmpb_plan_get_boxes.restype = I32
    lib.afmpb_plan_get_boxes.argtypes = [P, I32, P, P, P]
    lib.afmpb_plan_destroy.restype = I32
    lib.afmpb_plan_destroy.argtypes = [P]
    lib.afmpb_matvec_parts.restype = I32
    lib.afmpb_matvec_parts.argtypes = [P, P, P, I32]
    lib.afmpb_solve.restype = I32
    lib.afmpb_solve.argtypes = [P, P, P, C.POINTER(SolveInfo)]
    lib.afmpb_energy.restype = I32
    lib.afmpb_solve_batch.restype = I32
    lib.afmpb_solve_batch.argtypes = [C.POINTER(P), I32, C.POINTER(P), C.POINTER(P), C.POINTER(SolveInfo),
                                      C.POINTER(I32)]
    lib.afmpb_energy.argtypes = [P, C.POINTER(D)]
    lib.afmpb_energy_noalloc.restype = I32
    lib.afmpb_energy_noalloc.argtypes = [P, C.POINTER(D)]
    lib.afmpb_get_autotune.restype = I32
    lib.afmpb_get_autotune.argtypes = [P, C.POINTER(AutotuneReport)]
    lib.afmpb_selftest_bounded_wait.restype = I32
    lib.afmpb_selftest_bounded_wait.argtypes = [C.c_int, C.POINTER(C.c_int)]
    lib.afmpb_server_create.restype = I32
    lib.afmpb_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(P)]
    lib.afmpb_server_create_batched.restype = I32
    lib.afmpb_server_create_batched.argtypes = [C.c_size_t, C.c_int, C.c_int, C.c_int, C.POINTER(P)]
    lib.afmpb_server_submit.restype = I32
    lib.afmpb_server_submit.argtypes = [P, C.POINTER(Request), C.POINTER(I64)]
    lib.afmpb_server_poll.restype = I32
    lib.afmpb_server_poll.argtypes = [P, I64, C.POINTER(Result)]
    lib.afmpb_server_wait.restype = I32
    lib.afmpb_server_wait.argtypes = [P, I64, D, C.POINTER(Result)]
    lib.afmpb_server_get_info.restype = I32
    lib.afmpb_server_get_info.argtypes = [P, C.POINTER(ServerInfo)]
    lib.afmpb_server_destroy.restype = I32
    lib.afmpb_server_destroy.argtypes = [P]
    lib.afmpb_rhs.restype = I32
    lib.afmpb_rhs.argtypes = [P, P]
    lib.afmpb_get_geometry.restype = I32
    lib.afmpb_get_geometry.argtypes = [P, P, P, P]
    lib.afmpb_get_near.restype = I32
    lib.afmpb_get_near.argtypes = [P, P, P, P, P]
    lib.afmpb_get_tree.restype = I32
    lib.afmpb_get_tree.argtypes = [P] + [P] * 13
    lib.afmpb_get_info.restype = I32
    lib.afmpb_get_info.argtypes = [P, C.POINTER(Info)]
    lib.afmpb_destroy.restype = I32
    lib.afmpb_destroy.argtypes = [P]
    lib.afmpb_last_error.restype = C.c_char_p
    lib.afmpb_last_error.argtypes = [P]
    lib.afmpb_estimate_bytes.restype = C.c_size_t
    lib.afmpb_estimate_bytes.argtypes = [I64, I64, I32, C.POINTER(Options)]
    lib.afmpb_version.restype = C.c_char_p
    lib.afmpb_profile_product.restype = I32
    lib.afmpb_profile_product.argtypes = [P, I32, P, C.c_size_t, C.POINTER(Profile)]
    _lib = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    raise TypeError("expected a device pointer, a tensor or a numpy array")


def _np(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _check(rc, h=None):
    if rc != 0:
        msg = load(build=False).afmpb_last_error(h).decode(errors="replace")
        raise AfmpbError(rc, msg)


def version() -> str:
    return load().afmpb_version().decode()


def selftest_bounded_wait(spin_limit=1000) -> bool:
    """Runs a device wait that nothing satisfies with a bounded poll count; True when the
    wait gave up and reported it (the library's failure path for expired waits)."""
    e = C.c_int(0)
    _check(load().afmpb_selftest_bounded_wait(int(spin_limit), C.byref(e)), None)
    return bool(e.value)


def estimate_bytes(n_nodes, n_atoms, order=6, leaf_cap=0, restart=0, charge_fmm=0) -> int:
    o = Options(leaf_cap=leaf_cap, restart=restart, charge_fmm=charge_fmm)
    return int(load().afmpb_estimate_bytes(int(n_nodes), int(n_atoms), int(order), C.byref(o)))


class Handle:
    """One molecule on the GPU (afmpb_create ... afmpb_destroy)."""

    def __init__(self, xyz, tri, atoms=None, q=None, eps_in=1.0, eps_out=80.0, kappa=0.0,
                 order=6, tol=1e-6, leaf_cap=0, restart=0, max_restart=0, abs_tol=0.0,
                 precision=0, near_c=0.0, stream=None, max_level=0, normals=None, m2l_tol=0.0,
                 charge_fmm=0, orth=0, m2l_method=0):
        self._lib = load()
        self._xyz = _np(xyz, np.float64)
        self._tri = _np(tri, np.int32)
        self.n = int(self._xyz.shape[0])
        self._nrm = None if normals is None else _np(normals, np.float64)
        mesh = Mesh(self.n, int(self._tri.shape[0]), self._xyz.ctypes.data, self._tri.ctypes.data,
                     None if self._nrm is None else self._nrm.ctypes.data)
        ch = None
        if atoms is not None and q is not None:
            self._atoms = _np(np.atleast_2d(atoms), np.float64)
            self._q = _np(q, np.float64).ravel()
            ch = Charges(int(self._q.size), self._atoms.ctypes.data, self._q.ctypes.data)
        st = stream
        if st is not None and not isinstance(st, int):
            st = int(getattr(st, "cuda_stream", st))
        opt = Options(int(leaf_cap), int(restart), int(max_restart), float(abs_tol), int(precision),
                      float(near_c), st, int(max_level), float(m2l_tol), int(charge_fmm), int(orth),
                      int(m2l_method))
        h = C.c_void_p()
        rc = self._lib.afmpb_create(C.byref(mesh), None if ch is None else C.byref(ch),
                                    float(eps_in), float(eps_out), float(kappa), int(order),
                                    float(tol), C.byref(opt), C.byref(h))
        _check(rc, None)
        self.h = h.value

    @classmethod
    def for_molecule(cls, mol, **kw):
        return cls(mol.xyz, mol.tri, mol.atoms, mol.q, mol.eps_in, mol.eps_out, mol.kappa, **kw)

    # -- products ---------------------------------------------------------------------
    def matvec(self, x_dev, y_dev):
        _check(self._lib.afmpb_matvec(self.h, _ptr(x_dev), _ptr(y_dev)), self.h)

    def matvec_parts(self, x_dev, y_dev, parts):
        _check(self._lib.afmpb_matvec_parts(self.h, _ptr(x_dev), _ptr(y_dev), int(parts)), self.h)

    def matvec_host(self, x, y=None):
        """Host buffers: numpy arrays, or (pinned) CPU tensors / raw host pointers."""
        if isinstance(x, np.ndarray) or not (hasattr(x, "data_ptr") or isinstance(x, int)):
            x = _np(x, np.float32)
        if y is None:
            y = np.empty(2 * self.n, np.float32)
        _check(self._lib.afmpb_matvec_host(self.h, _ptr(x), _ptr(y)), self.h)
        return y

    def sync(self):
        """Wait for the handle's stream; raises ETIMEOUT if a bounded device wait expired."""
        _check(self._lib.afmpb_sync(self.h), self.h)

    def inject_wait_expiry(self):
        """Test hook: set the handle's bounded-wait flag from the host (no device fault)."""
        _check(self._lib.afmpb_inject_wait_expiry(self.h), self.h)

    def profile(self, reps=5, flush=None, flush_bytes=0):
        """Per-stage product timings (ms) measured with CUDA events in the library."""
        p = Profile()
        _check(self._lib.afmpb_profile_product(self.h, int(reps), _ptr(flush), int(flush_bytes),
                                               C.byref(p)), self.h)
        stages = [(p.name[i].value.decode(), p.ms[i], p.launches[i]) for i in range(p.n_stages)]
        return dict(stages=stages, ms_graph=p.ms_graph, kernels_per_product=p.kernels_per_product)

    # -- solve --------------------------------------------------------------------------
    def solve(self, raise_on_noconv=True):
        f = np.zeros(self.n)
        hh = np.zeros(self.n)
        info = SolveInfo()
        rc = self._lib.afmpb_solve(self.h, f.ctypes.data, hh.ctypes.data, C.byref(info))
        d = _struct_dict(info)
        d["status"] = STATUS.get(rc, rc)
        if rc != 0 and (rc != 5 or raise_on_noconv):
            _check(rc, self.h)
        return f, hh, d

    def energy(self):
        e = C.c_double()
        _check(self._lib.afmpb_energy(self.h, C.byref(e)), self.h)
        return float(e.value)

    def energy_noalloc(self):
        """Same energy as energy(), computed without any device allocation (static scratch)."""
        e = C.c_double()
        _check(self._lib.afmpb_energy_noalloc(self.h, C.byref(e)), self.h)
        return float(e.value)

    def rhs(self):
        b = np.zeros(2 * self.n)
        _check(self._lib.afmpb_rhs(self.h, b.ctypes.data), self.h)
        return b

    # -- exports ------------------------------------------------------------------------
    def info(self):
        i = Info()
        _check(self._lib.afmpb_get_info(self.h, C.byref(i)), self.h)
        return _struct_dict(i)

    def autotune(self):
        """The leaf-capacity tuner's report (None unless this handle ran the tuner)."""
        r = AutotuneReport()
        rc = self._lib.afmpb_get_autotune(self.h, C.byref(r))
        if rc == 8:
            return None
        _check(rc, self.h)
        k = r.n_candidates
        d = _struct_dict(r)
        for key in ("cap", "p2p_ms", "predicted_ms"):
            d[key] = d[key][:k]
        return d

    def geometry(self):
        a = np.zeros(self.n)
        nrm = np.zeros((self.n, 3))
        rho = np.zeros(self.n)
        _check(self._lib.afmpb_get_geometry(self.h, a.ctypes.data, nrm.ctypes.data, rho.ctypes.data), self.h)
        return a, nrm, rho

    def near(self):
        nnz = self.info()["nnz_near"]
        rp = np.zeros(self.n + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        coef = np.zeros((nnz, 4), np.float32)
        whole = np.zeros(nnz, np.uint8)
        _check(self._lib.afmpb_get_near(self.h, rp.ctypes.data, col.ctypes.data, coef.ctypes.data,
                                        whole.ctypes.data), self.h)
        return rp, col, coef, whole.astype(bool)

    def tree(self):
        inf = self.info()
        nb = inf["n_boxes"]
        t = dict(level=np.zeros(nb, np.int32), anchor=np.zeros((nb, 3), np.int32),
                 range=np.zeros((nb, 2), np.int32), parent=np.zeros(nb, np.int32),
                 perm=np.zeros(self.n, np.int32))
        for k, key in (("u", "n_list_u"), ("v", "n_list_v"), ("w", "n_list_w"), ("x", "n_list_x")):
            t[k + "_ptr"] = np.zeros(nb + 1, np.int64)
            t[k + "_idx"] = np.zeros(max(1, inf[key]), np.int32)
        args = [t["level"], t["anchor"], t["range"], t["parent"], t["perm"],
                t["u_ptr"], t["u_idx"], t["v_ptr"], t["v_idx"], t["w_ptr"], t["w_idx"],
                t["x_ptr"], t["x_idx"]]
        _check(self._lib.afmpb_get_tree(self.h, *[a.ctypes.data for a in args]), self.h)
        for k, key in (("u", "n_list_u"), ("v", "n_list_v"), ("w", "n_list_w"), ("x", "n_list_x")):
            t[k + "_idx"] = t[k + "_idx"][: inf[key]]
        return t

    def close(self):
        if getattr(self, "h", None):
            self._lib.afmpb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


BATCH_MAX = 64


def solve_batch(handles, raise_on_noconv=True):
    """Solves the problems of several handles together (afmpb_solve_batch): lockstep GMRES
    with one fused P2P and one fused tensor-core M2L launch per Arnoldi step.  Returns one
    (f, h, info) per handle, as Handle.solve does, info["status"] per problem."""
    lib = load(build=False)
    k = len(handles)
    hs = (C.c_void_p * k)(*[h.h for h in handles])
    fs = [np.zeros(h.n) for h in handles]
    hh = [np.zeros(h.n) for h in handles]
    fp = (C.c_void_p * k)(*[a.ctypes.data for a in fs])
    hp = (C.c_void_p * k)(*[a.ctypes.data for a in hh])
    infos = (SolveInfo * k)()
    st = (C.c_int * k)()
    rc = lib.afmpb_solve_batch(hs, k, fp, hp, infos, st)
    out = []
    for i in range(k):
        d = _struct_dict(infos[i])
        d["status"] = STATUS.get(st[i], st[i]) if rc in (0, 5, 6) else STATUS.get(rc, rc)
        out.append((fs[i], hh[i], d))
    if rc != 0 and (rc != 5 or raise_on_noconv):
        _check(rc, handles[0].h if k else None)
    return out


def plan_partition(tree, n_nodes, nranks, near_ptr=None, near_col=None):
    """The multi-GPU partition plan of one solve (afmpb_plan_*): host-side planning only.
    tree: dict with range [nb, 2], parent [nb] and u/v/w/x _ptr/_idx arrays (the layout of
    Handle.tree()); near_ptr / near_col: optional near-field CSR over Morton positions.
    Returns one dict per rank: node range, work, halo nodes and owners, send nodes and
    destinations, imported list-2 boxes and owners (-1 shared), shared boxes."""
    lib = load()
    keep = {}

    def arr(name, a, dt):
        keep[name] = _np(a, dt)
        return keep[name].ctypes.data

    nb = int(np.asarray(tree["parent"]).shape[0])
    pin = PlanInput(int(n_nodes), nb, arr("range", tree["range"], np.int32), arr("parent", tree["parent"], np.int32),
                    arr("u_ptr", tree["u_ptr"], np.int64), arr("u_idx", tree["u_idx"], np.int32),
                    arr("v_ptr", tree["v_ptr"], np.int64), arr("v_idx", tree["v_idx"], np.int32),
                    arr("w_ptr", tree["w_ptr"], np.int64), arr("w_idx", tree["w_idx"], np.int32),
                    arr("x_ptr", tree["x_ptr"], np.int64), arr("x_idx", tree["x_idx"], np.int32),
                    None if near_ptr is None else arr("near_ptr", near_ptr, np.int64),
                    None if near_col is None else arr("near_col", near_col, np.int32))
    p = C.c_void_p()
    rc = lib.afmpb_plan_create(C.byref(pin), int(nranks), C.byref(p))
    if rc != 0:
        raise AfmpbError(rc, "afmpb_plan_create")
    out = []
    try:
        for r in range(nranks):
            info = PlanRank()
            _check(lib.afmpb_plan_get_rank(p, r, C.byref(info)))
            d = _struct_dict(info)
            d["halo"] = np.zeros(info.n_halo, np.int64)
            d["halo_owner"] = np.zeros(info.n_halo, np.int32)
            d["send"] = np.zeros(info.n_send, np.int64)
            d["send_dest"] = np.zeros(info.n_send, np.int32)
            d["imports"] = np.zeros(info.n_import_boxes, np.int32)
            d["import_owner"] = np.zeros(info.n_import_boxes, np.int32)
            d["shared"] = np.zeros(info.n_shared_boxes, np.int32)
            _check(lib.afmpb_plan_get_halo(p, r, d["halo"].ctypes.data, d["halo_owner"].ctypes.data))
            _check(lib.afmpb_plan_get_send(p, r, d["send"].ctypes.data, d["send_dest"].ctypes.data))
            _check(lib.afmpb_plan_get_boxes(p, r, d["imports"].ctypes.data, d["import_owner"].ctypes.data,
                                            d["shared"].ctypes.data))
            out.append(d)
    finally:
        lib.afmpb_plan_destroy(p)
    return out


def _result_dict(r):
    d = {"status": STATUS.get(r.status, r.status), "error": r.error.decode(errors="replace"),
         "energy": r.energy_kcal_mol, "info": _struct_dict(r.info), "t_submit": r.t_submit,
         "t_admit": r.t_admit, "t_done": r.t_done, "bytes_reserved": r.bytes_reserved,
         "bytes_used": r.bytes_used, "slot": r.slot}
    d["latency"] = r.t_done - r.t_submit
    return d


class Server:
    """Continuous-batching solve server (afmpb_server_*): submit whole solves, poll or wait
    for their results; requests overlap on the GPU as slots and device memory allow."""

    def __init__(self, bytes_budget, max_slots=4, max_batch=1, solvers=1):
        self._lib = load()
        h = C.c_void_p()
        rc = self._lib.afmpb_server_create_batched(int(bytes_budget), int(max_slots), int(solvers), int(max_batch),
                                                   C.byref(h))
        if rc != 0:
            raise AfmpbError(rc, "afmpb_server_create failed")
        self.s = h.value
        self._keep = {}          # ticket -> output buffers that the server writes into

    def submit(self, xyz, tri, atoms, q, eps_in=1.0, eps_out=80.0, kappa=0.0, order=6, tol=1e-6,
               precision=0, leaf_cap=0, m2l_tol=0.0, restart=0, max_restart=0, want_solution=False,
               charge_fmm=0, orth=0):
        xyz = _np(xyz, np.float64)
        tri = _np(tri, np.int32)
        atoms = _np(np.atleast_2d(atoms), np.float64)
        q = _np(q, np.float64).ravel()
        n = int(xyz.shape[0])
        f = np.zeros(n) if want_solution else None
        hh = np.zeros(n) if want_solution else None
        req = Request(Mesh(n, int(tri.shape[0]), xyz.ctypes.data, tri.ctypes.data, None),
                      Charges(int(q.size), atoms.ctypes.data, q.ctypes.data),
                      float(eps_in), float(eps_out), float(kappa), int(order), float(tol),
                      Options(int(leaf_cap), int(restart), int(max_restart), 0.0, int(precision), 0.0, None, 0,
                              float(m2l_tol), int(charge_fmm), int(orth)),
                      None if f is None else f.ctypes.data, None if hh is None else hh.ctypes.data)
        t = C.c_int64()
        rc = self._lib.afmpb_server_submit(self.s, C.byref(req), C.byref(t))
        if rc != 0:
            raise AfmpbError(rc, "afmpb_server_submit refused the request")
        self._keep[t.value] = (f, hh)
        return t.value

    def submit_molecule(self, mol, **kw):
        return self.submit(mol.xyz, mol.tri, mol.atoms, mol.q, mol.eps_in, mol.eps_out, mol.kappa, **kw)

    def _finish(self, ticket, r):
        d = _result_dict(r)
        f, hh = self._keep.pop(ticket, (None, None))
        if f is not None:
            d["f"], d["h"] = f, hh
        return d

    def poll(self, ticket):
        """The result dict, or None while the request is pending."""
        r = Result()
        rc = self._lib.afmpb_server_poll(self.s, int(ticket), C.byref(r))
        if rc == 7:
            return None
        if rc != 0:
            raise AfmpbError(rc, "afmpb_server_poll")
        return self._finish(ticket, r)

    def wait(self, ticket, timeout=600.0):
        r = Result()
        rc = self._lib.afmpb_server_wait(self.s, int(ticket), float(timeout), C.byref(r))
        if rc != 0:
            raise AfmpbError(rc, "afmpb_server_wait")
        return self._finish(ticket, r)

    def info(self):
        i = ServerInfo()
        _check(self._lib.afmpb_server_get_info(self.s, C.byref(i)))
        return _struct_dict(i)

    def close(self):
        if getattr(self, "s", None):
            self._lib.afmpb_server_destroy(self.s)
            self.s = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
