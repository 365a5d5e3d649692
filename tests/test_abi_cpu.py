"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/afmpb.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "afmpb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(afmpb_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("afmpb_create", "afmpb_matvec", "afmpb_solve", "afmpb_energy", "afmpb_destroy"):
        assert s in syms


def test_library_builds_and_exports_every_declared_symbol():
    import paper_1710_06316_gb300 as pb
    lib = pb.load()
    assert os.path.exists(pb.library_path())
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert set(declared_symbols()) == set(pb.EXPORTS)


def test_host_only_entry_points():
    import paper_1710_06316_gb300 as pb
    assert "sm_103a" in pb.version()
    b1 = pb.estimate_bytes(2562, 1)
    b2 = pb.estimate_bytes(163842, 64)
    assert 0 < b1 < b2
    # the charge FMM (forced, or above the pair threshold) adds its octree to the estimate
    assert pb.estimate_bytes(163842, 64, charge_fmm=2) > b2
    assert pb.estimate_bytes(163842, 64, charge_fmm=1) == b2
    big = pb.estimate_bytes(10_000_000, 1_200_000, charge_fmm=1)
    assert pb.estimate_bytes(10_000_000, 1_200_000) > big
    lib = pb.load()
    assert lib.afmpb_estimate_bytes(0, 0, 6, None) == 0          # invalid size
    assert lib.afmpb_estimate_bytes(100, 0, 9, None) == 0        # invalid order


def test_null_arguments_are_rejected_without_a_device():
    import paper_1710_06316_gb300 as pb
    lib = pb.load()
    out = ctypes.c_void_p()
    # NULL mesh -> EINVAL before any CUDA call
    rc = lib.afmpb_create(None, None, 1.0, 80.0, 0.1, 6, 1e-6, None, ctypes.byref(out))
    assert rc == 1 and out.value is None
    assert b"mesh" in lib.afmpb_last_error(None)
    assert lib.afmpb_matvec(None, None, None) == 1
    assert lib.afmpb_sync(None) == 1
    assert lib.afmpb_inject_wait_expiry(None) == 1
    # batched solve: no handles, too many, or a NULL handle -> EINVAL on the host
    assert lib.afmpb_solve_batch(None, 1, None, None, None, None) == 1
    hs = (ctypes.c_void_p * 2)(None, None)
    assert lib.afmpb_solve_batch(hs, 0, None, None, None, None) == 1
    assert lib.afmpb_solve_batch(hs, 65, None, None, None, None) == 1
    assert lib.afmpb_solve_batch(hs, 2, None, None, None, None) == 1
    assert lib.afmpb_destroy(None) == 0


def test_invalid_mesh_is_rejected_on_the_host():
    """Mesh validation runs before any device work, so it is testable on CPU."""
    import numpy as np
    import paper_1710_06316_gb300 as pb
    import synthetic
    xyz, tri = synthetic.icosphere(2)
    bad = tri[1:]                      # open surface
    with pytest.raises(pb.AfmpbError) as e:
        pb.Handle(xyz, bad, eps_in=1, eps_out=80, kappa=0.1)
    assert e.value.status == "EMESH"
    with pytest.raises(pb.AfmpbError) as e:
        pb.Handle(xyz, tri[:, [0, 2, 1]], eps_in=1, eps_out=80, kappa=0.1)   # inward
    assert e.value.status == "EMESH"
    with pytest.raises(pb.AfmpbError) as e:
        pb.Handle(xyz, tri, eps_in=-1, eps_out=80, kappa=0.1)
    assert e.value.status == "EINVAL"
    with pytest.raises(pb.AfmpbError) as e:
        pb.Handle(xyz, tri, eps_in=1, eps_out=80, kappa=0.1, order=9)
    assert e.value.status == "EINVAL"
    with pytest.raises(pb.AfmpbError) as e:
        pb.Handle(xyz, tri, eps_in=1, eps_out=80, kappa=0.1, charge_fmm=3)
    assert e.value.status == "EINVAL"
    xyz2 = xyz.copy()
    xyz2[3, 0] = np.nan
    with pytest.raises(pb.AfmpbError) as e:
        pb.Handle(xyz2, tri, eps_in=1, eps_out=80, kappa=0.1)
    assert e.value.status == "EINVAL"


def test_selftest_arguments_are_checked_on_the_host():
    import ctypes
    import paper_1710_06316_gb300 as pb
    lib = pb.load()
    e = ctypes.c_int(7)
    assert lib.afmpb_selftest_bounded_wait(0, ctypes.byref(e)) == 1        # EINVAL
    assert lib.afmpb_selftest_bounded_wait(100, None) == 1
    assert lib.afmpb_selftest_bounded_wait((1 << 26) + 1, ctypes.byref(e)) == 1


_GOOD = dict(eps_in=2.0, eps_out=80.0, kappa=0.1, order=6, tol=1e-6)
_BAD_ARGS = [
    ("eps_in zero", dict(eps_in=0.0), b"eps_in"),
    ("eps_out infinite", dict(eps_out=float("inf")), b"eps_in"),
    ("kappa negative", dict(kappa=-0.1), b"kappa"),
    ("kappa NaN", dict(kappa=float("nan")), b"kappa"),
    ("order 1", dict(order=1), b"fmm_order"),
    ("tol zero", dict(tol=0.0), b"tol"),
    ("tol NaN", dict(tol=float("nan")), b"tol"),
]
_BAD_OPTIONS = [
    ("negative restart", dict(restart=-2), b"negative option"),
    ("unknown orthogonalisation", dict(orth=2), b"orth"),
    ("restart above 4096", dict(restart=4097), b"restart"),
    ("negative max_restart", dict(max_restart=-2), b"negative option"),
    ("negative leaf cap", dict(leaf_cap=-5), b"negative option"),
    ("max_level 21", dict(max_level=21), b"max_level"),
    ("negative abs_tol", dict(abs_tol=-1e-9), b"abs_tol"),
    ("NaN near_c", dict(near_c=float("nan")), b"near_c"),
    ("precision 2", dict(precision=2), b"precision"),
    ("charge_fmm -1", dict(charge_fmm=-1), b"charge_fmm"),
    ("unknown M2L method", dict(m2l_method=2), b"m2l_method"),
]


def _create(args=None, options=None, charges=None):
    import numpy as np
    import paper_1710_06316_gb300 as pb
    import synthetic
    lib = pb.load()
    xyz, tri = synthetic.icosphere(1)
    xyz = np.ascontiguousarray(xyz, np.float64)
    tri = np.ascontiguousarray(tri, np.int32)
    mesh = pb.Mesh(xyz.shape[0], tri.shape[0], xyz.ctypes.data, tri.ctypes.data, None)
    a = dict(_GOOD, **(args or {}))
    opt = None
    if options is not None:
        opt = pb.Options()
        for k, v in options.items():
            setattr(opt, k, v)
    out = ctypes.c_void_p()
    rc = lib.afmpb_create(ctypes.byref(mesh), None if charges is None else ctypes.byref(charges),
                          a["eps_in"], a["eps_out"], a["kappa"], a["order"], a["tol"],
                          None if opt is None else ctypes.byref(opt), ctypes.byref(out))
    return rc, out.value, lib.afmpb_last_error(None)


@pytest.mark.parametrize("what,args,word", _BAD_ARGS, ids=[b[0] for b in _BAD_ARGS])
def test_invalid_scalar_arguments_are_rejected_on_the_host(what, args, word):
    rc, handle, msg = _create(args=args)
    assert rc == 1 and handle is None      # EINVAL, no handle, before any CUDA call
    assert word in msg, msg


@pytest.mark.parametrize("what,opts,word", _BAD_OPTIONS, ids=[b[0] for b in _BAD_OPTIONS])
def test_invalid_options_are_rejected_on_the_host(what, opts, word):
    rc, handle, msg = _create(options=opts)
    assert rc == 1 and handle is None
    assert word in msg, msg


def test_invalid_charges_are_rejected_on_the_host():
    import paper_1710_06316_gb300 as pb
    rc, handle, msg = _create(charges=pb.Charges(3, None, None))
    assert rc == 1 and handle is None and b"charges" in msg
    rc, handle, msg = _create(charges=pb.Charges(-1, None, None))
    assert rc == 1 and handle is None and b"charges" in msg
