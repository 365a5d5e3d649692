"""The host-side node -> triangle-corner buckets (csrc/corner_csr.h) used by the mesh
check and the geometry setup: the parallel two-level counting sort gives, for every
thread count, exactly the buckets of a stable sort of the corners by node.  The header
is plain C++; it is compiled here with g++ (no CUDA, no GPU)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "paper_1710_06316_gb300", "csrc")

DRIVER = r"""
#include <cstring>
#include "corner_csr.h"
extern "C" void corners(int64_t n, int64_t nt, const int32_t *tri, int threads, int next_node,
                        int64_t *ptr, int32_t *out) {
  std::unique_ptr<int64_t[]> p;
  std::unique_ptr<int32_t[]> o;
  if (next_node)
    afmpb::corner_csr(n, nt, tri, threads, p, o, [tri](int64_t t, int k) { return tri[3 * t + (k + 1) % 3]; });
  else
    afmpb::corner_csr(n, nt, tri, threads, p, o, [](int64_t t, int) { return (int32_t)t; });
  std::memcpy(ptr, p.get(), sizeof(int64_t) * (n + 1));
  std::memcpy(out, o.get(), sizeof(int32_t) * 3 * nt);
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("corner_csr")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    so = d / "libcorners.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-fPIC", "-shared", "-I", HEADER_DIR,
                           str(src), "-o", str(so)])
    L = ctypes.CDLL(str(so))
    L.corners.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                          ctypes.c_void_p, ctypes.c_void_p]
    return L


def reference(n, tri, next_node):
    node = tri.ravel()
    t = np.repeat(np.arange(tri.shape[0]), 3)
    k = np.tile(np.arange(3), tri.shape[0])
    value = tri[t, (k + 1) % 3] if next_node else t
    order = np.argsort(node, kind="stable")       # ties keep corner order: t, then k
    ptr = np.concatenate([[0], np.cumsum(np.bincount(node, minlength=n))])
    return ptr, value[order].astype(np.int32)


@pytest.mark.parametrize("n,nt", [(5, 4), (4096, 3000), (4097, 9000), (20000, 1), (70001, 150000)])
def test_buckets_equal_a_stable_sort_for_every_thread_count(lib, n, nt):
    rng = np.random.default_rng(n + nt)
    # clustered indices (like a mesh) with some nodes unused
    base = rng.integers(0, n, nt)
    tri = np.clip(base[:, None] + rng.integers(-40, 40, (nt, 3)), 0, n - 1).astype(np.int32)
    for next_node in (1, 0):
        ptr_ref, out_ref = reference(n, tri, next_node)
        for threads in (1, 2, 3, 8, 16):
            ptr = np.empty(n + 1, np.int64)
            out = np.empty(3 * nt, np.int32)
            lib.corners(n, nt, tri.ctypes.data, threads, next_node, ptr.ctypes.data, out.ctypes.data)
            assert np.array_equal(ptr, ptr_ref), (threads, next_node)
            assert np.array_equal(out, out_ref), (threads, next_node)
