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
