"""One solve on several GPUs: the partition plan (afmpb_plan_*), host-side.

The fixture builds a small adaptive octree over an icosphere's nodes in numpy -- boxes
split while they hold more than `cap` nodes, lists 1-4 by their definitions (Carrier,
Greengard and Rokhlin; list 3 evaluated point to point as the paper's modified method
does, Sec. 3.2) by brute force over box pairs -- and a near-field CSR by a radius rule.
The plan must
  * cut the Morton order between leaves into ranges that tile the nodes, with balanced work;
  * give every rank exactly the outside source nodes its rows read (halo), with owners,
    and send lists that are the transpose of the halos;
  * list every list-2 source box of the rank's boxes that is not inside its range.
Then three gloo ranks on the CPU run a distributed product (each rank: its rows; the halo
exchanged by all-to-all as the plan says) and a distributed GMRES whose Krylov vectors are
split like the nodes (inner products by all-reduce), against the single-process result.
"""
import os
import socket
import sys

import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# ---- fixture: adaptive octree and lists in numpy ------------------------------------------
def build_tree(pts, cap):
    lo = pts.min(0)
    w = (pts.max(0) - lo).max() * 1.000001
    q = np.floor((pts - lo) / w * (1 << 10)).astype(np.int64)
    key = np.zeros(len(pts), np.int64)
    for bit in range(10):
        for d in range(3):
            key |= ((q[:, d] >> bit) & 1) << (3 * bit + (2 - d))
    order = np.argsort(key, kind="stable")
    key = key[order]
    boxes = [dict(level=0, anchor=(0, 0, 0), lo=0, hi=len(pts), parent=-1)]
    i = 0
    while i < len(boxes):
        b = boxes[i]
        if b["hi"] - b["lo"] > cap and b["level"] < 9:
            lvl = b["level"] + 1
            shift = 3 * (10 - lvl)
            seg = key[b["lo"]:b["hi"]] >> shift
            for o in range(8):
                code = (_code(b["anchor"], b["level"]) << 3) | o
                s = b["lo"] + np.searchsorted(seg, code, "left")
                e = b["lo"] + np.searchsorted(seg, code, "right")
                if e > s:
                    a = tuple(2 * b["anchor"][d] + ((o >> (2 - d)) & 1) for d in range(3))
                    boxes.append(dict(level=lvl, anchor=a, lo=int(s), hi=int(e), parent=i))
        i += 1
    nb = len(boxes)
    children = [[] for _ in range(nb)]
    for k, b in enumerate(boxes):
        if b["parent"] >= 0:
            children[b["parent"]].append(k)
    leaf = [not c for c in children]

    def adjacent(a, b):
        A, B = boxes[a], boxes[b]
        if A["level"] > B["level"]:
            A, B = B, A
        s = B["level"] - A["level"]
        return all(B["anchor"][d] + 1 >= A["anchor"][d] << s and B["anchor"][d] <= (A["anchor"][d] + 1) << s
                   for d in range(3))

    U, V, W, X = ([[] for _ in range(nb)] for _ in range(4))
    for b in range(nb):
        if boxes[b]["parent"] >= 0:
            p = boxes[b]["parent"]
            for c in range(nb):          # list 2: children of the parent's colleagues, not adjacent
                if boxes[c]["level"] == boxes[b]["level"] and boxes[c]["parent"] >= 0 and \
                        adjacent(boxes[c]["parent"], p) and boxes[boxes[c]["parent"]]["level"] == boxes[p]["level"] \
                        and not adjacent(b, c):
                    V[b].append(c)
        if not leaf[b]:
            continue
        for c in range(nb):
            if leaf[c] and adjacent(b, c):
                U[b].append(c)           # list 1: adjacent leaves
            if boxes[c]["parent"] >= 0 and not adjacent(b, c) and adjacent(b, boxes[c]["parent"]) \
                    and boxes[c]["level"] > boxes[b]["level"]:
                W[b].append(c)           # list 3
    for b in range(nb):
        for c in W[b]:
            X[c].append(b)               # list 4: the dual of list 3

    def csr(lists):
        ptr = np.zeros(nb + 1, np.int64)
        ptr[1:] = np.cumsum([len(l) for l in lists])
        idx = np.array([c for l in lists for c in sorted(l)], np.int32)
        return ptr, idx

    t = {"range": np.array([[b["lo"], b["hi"]] for b in boxes], np.int32),
         "parent": np.array([b["parent"] for b in boxes], np.int32), "leaf": np.array(leaf)}
    for name, lists in (("u", U), ("v", V), ("w", W), ("x", X)):
        t[name + "_ptr"], t[name + "_idx"] = csr(lists)
    return t, order


def _code(anchor, level):
    c = 0
    for bit in range(level):
        for d in range(3):
            c |= ((anchor[d] >> bit) & 1) << (3 * bit + (2 - d))
    return c


def near_csr(p, radius):
    n = len(p)
    d = np.linalg.norm(p[:, None, :] - p[None, :, :], axis=2)
    rows = [np.nonzero(d[i] < radius)[0] for i in range(n)]
    ptr = np.zeros(n + 1, np.int64)
    ptr[1:] = np.cumsum([len(r) for r in rows])
    return ptr, np.concatenate(rows).astype(np.int32)


@pytest.fixture(scope="module")
def sphere_tree():
    xyz, _ = synthetic.icosphere(3, radius=10.0)        # 642 nodes
    tree, order = build_tree(xyz, cap=12)
    p = xyz[order]
    nptr, ncol = near_csr(p, 2.2)
    return p, tree, nptr, ncol


def sources_of_rows(tree, nptr, ncol, a, e, n):
    """Every source node the rows [a, e) read: lists 1, 3 of their leaves, list 4 of boxes
    touching the range, near-field columns."""
    need = np.zeros(n, bool)
    rng, par = tree["range"], tree["parent"]
    for b in range(len(par)):
        lo, hi = rng[b]
        if hi <= a or lo >= e:
            continue
        if tree["leaf"][b]:
            for name in ("u", "w"):
                for c in tree[name + "_idx"][tree[name + "_ptr"][b]:tree[name + "_ptr"][b + 1]]:
                    need[rng[c, 0]:rng[c, 1]] = True
        for c in tree["x_idx"][tree["x_ptr"][b]:tree["x_ptr"][b + 1]]:
            need[rng[c, 0]:rng[c, 1]] = True
    for t in range(a, e):
        need[ncol[nptr[t]:nptr[t + 1]]] = True
    need[a:e] = False
    return np.nonzero(need)[0]


# ---- the plan itself ------------------------------------------------------------------------
@pytest.mark.parametrize("nranks", [1, 2, 3, 5])
def test_plan_ranges_halos_and_imports(sphere_tree, nranks):
    import paper_1710_06316_gb300 as pb
    p, tree, nptr, ncol = sphere_tree
    n = len(p)
    plan = pb.plan_partition(tree, n, nranks, nptr, ncol)
    leaf_starts = set(tree["range"][tree["leaf"], 0].tolist()) | {n}
    assert plan[0]["node_begin"] == 0 and plan[-1]["node_end"] == n
    for r in range(nranks):
        assert plan[r]["node_begin"] <= plan[r]["node_end"]
        if r:
            assert plan[r]["node_begin"] == plan[r - 1]["node_end"]
        assert plan[r]["node_begin"] in leaf_starts           # cuts between leaves only
    work = np.array([d["work"] for d in plan])
    assert work.max() <= 1.6 * work.mean() + 1e-9
    for r, d in enumerate(plan):
        want = sources_of_rows(tree, nptr, ncol, d["node_begin"], d["node_end"], n)
        np.testing.assert_array_equal(d["halo"], want)
        for t, o in zip(d["halo"], d["halo_owner"]):
            assert plan[o]["node_begin"] <= t < plan[o]["node_end"]
        # every list-2 source of a box touching the range, not inside it, is imported
        rng = tree["range"]
        need = set()
        for b in range(len(rng)):
            if rng[b, 1] <= d["node_begin"] or rng[b, 0] >= d["node_end"]:
                continue
            for c in tree["v_idx"][tree["v_ptr"][b]:tree["v_ptr"][b + 1]]:
                if not (rng[c, 0] >= d["node_begin"] and rng[c, 1] <= d["node_end"]):
                    need.add(int(c))
        assert set(d["imports"].tolist()) == need
        for c, o in zip(d["imports"], d["import_owner"]):
            lo, hi = rng[c]
            if o >= 0:
                assert plan[o]["node_begin"] <= lo and hi <= plan[o]["node_end"]
            else:
                assert any(plan[q]["node_begin"] <= lo < plan[q]["node_end"] for q in range(nranks))
    # send lists are the transpose of the halos
    sent = sorted((int(t), int(dst)) for d in plan for t, dst in zip(d["send"], d["send_dest"]))
    recv = sorted((int(t), r) for r, d in enumerate(plan) for t in d["halo"])
    assert sent == recv
    if nranks == 1:
        assert plan[0]["n_halo"] == 0 and plan[0]["n_import_boxes"] == 0


def test_plan_rejects_bad_input():
    import ctypes
    import paper_1710_06316_gb300 as pb
    lib = pb.load()
    out = ctypes.c_void_p()
    assert lib.afmpb_plan_create(None, 2, ctypes.byref(out)) == 1
    tree = dict(range=np.array([[0, 5]], np.int32), parent=np.array([-1], np.int32))
    for k in "uvwx":
        tree[k + "_ptr"] = np.zeros(2, np.int64)
        tree[k + "_idx"] = np.zeros(1, np.int32)
    with pytest.raises(pb.AfmpbError):
        pb.plan_partition(tree, 4, 2)                        # box range beyond n_nodes
    with pytest.raises(pb.AfmpbError):
        pb.plan_partition(tree, 5, 0)


# ---- three gloo ranks: distributed product and GMRES ---------------------------------------
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _operator(p, tree, nptr, ncol):
    """A test operator with the product's sparsity: near-field entries plus point pairs of
    lists 1, 3, 4 (rows in Morton order); A = I + 0.02 * K."""
    n = len(p)
    K = np.zeros((n, n))
    rng = tree["range"]
    for b in range(len(rng)):
        rows = range(rng[b, 0], rng[b, 1])
        cols = []
        if tree["leaf"][b]:
            for name in ("u", "w"):
                for c in tree[name + "_idx"][tree[name + "_ptr"][b]:tree[name + "_ptr"][b + 1]]:
                    cols.extend(range(rng[c, 0], rng[c, 1]))
            a = b
            while a >= 0:
                for c in tree["x_idx"][tree["x_ptr"][a]:tree["x_ptr"][a + 1]]:
                    cols.extend(range(rng[c, 0], rng[c, 1]))
                a = tree["parent"][a]
            for i in rows:
                for j in cols:
                    if i != j:
                        K[i, j] = 1.0 / (1.0 + np.linalg.norm(p[i] - p[j]))
    for i in range(n):
        for j in ncol[nptr[i]:nptr[i + 1]]:
            K[i, j] += 0.5 * np.sin(i + 2.0 * j)
    return np.eye(n) + 0.02 * K


def _rank_main(rank, world, port, data, out):
    sys.path.insert(0, ROOT)
    import paper_1710_06316_gb300 as pb
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, tree, nptr, ncol, A, b = data
        n = len(p)
        plan = pb.plan_partition(tree, n, world, nptr, ncol)
        me = plan[rank]
        a, e = me["node_begin"], me["node_end"]
        halo = me["halo"]

        def exchange(x_own):
            """x values of this rank's halo, received from their owners (all-to-all)."""
            send_nodes, dest = me["send"], me["send_dest"]
            counts_out = [int((dest == q).sum()) for q in range(world)]
            counts_in = [int((me["halo_owner"] == q).sum()) for q in range(world)]
            send_buf = torch.tensor(x_own[send_nodes - a], dtype=torch.float64)
            recv_buf = torch.empty(len(halo), dtype=torch.float64)
            dist.all_to_all_single(recv_buf, send_buf, counts_in, counts_out)
            # received in owner order; halo is ascending and owners are ascending ranges
            return recv_buf.numpy()

        def product(x_own):
            xh = exchange(x_own)
            cols = np.concatenate([np.arange(a, e), halo])
            vals = np.concatenate([x_own, xh])
            return A[a:e][:, cols] @ vals           # only the columns the plan delivered

        def dot(u, v):
            t = torch.tensor([float(u @ v)], dtype=torch.float64)
            dist.all_reduce(t)
            return float(t.item())

        # the product against the single-process one
        x = np.sin(np.arange(n) * 0.37)
        y_rank = product(x[a:e])
        # distributed GMRES(30): Krylov vectors split like the nodes, inner products all-reduced
        m = 30
        bl = b[a:e]
        xl = np.zeros(e - a)
        bn = np.sqrt(dot(bl, bl))
        for _ in range(10):
            r = bl - product(xl)
            beta = np.sqrt(dot(r, r))
            if beta <= 1e-10 * bn:
                break
            Vl = [r / beta]
            H = np.zeros((m + 1, m))
            k = m
            for j in range(m):
                w = product(Vl[j])
                for i in range(j + 1):              # modified Gram-Schmidt, all-reduced dots
                    H[i, j] = dot(w, Vl[i])
                    w = w - H[i, j] * Vl[i]
                H[j + 1, j] = np.sqrt(dot(w, w))
                if H[j + 1, j] < 1e-14:
                    k = j + 1
                    break
                Vl.append(w / H[j + 1, j])
            g = np.zeros(k + 1)
            g[0] = beta
            yk = np.linalg.lstsq(H[:k + 1, :k], g, rcond=None)[0]
            xl = xl + np.stack(Vl[:k], 1) @ yk
        out[rank] = (a, e, y_rank, xl)
    finally:
        dist.destroy_process_group()


def test_three_gloo_ranks_product_and_gmres_match_one_process(sphere_tree):
    p, tree, nptr, ncol = sphere_tree
    n = len(p)
    A = _operator(p, tree, nptr, ncol)
    b = np.cos(np.arange(n) * 0.11)
    x = np.sin(np.arange(n) * 0.37)
    y_ref = A @ x
    x_ref = np.linalg.solve(A, b)
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    world = 3
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, (p, tree, nptr, ncol, A, b), out))
             for r in range(world)]
    for q in procs:
        q.start()
    for q in procs:
        q.join(300)
        assert q.exitcode == 0
    y = np.zeros(n)
    xs = np.zeros(n)
    for r in range(world):
        a, e, yr, xr = out[r]
        y[a:e] = yr
        xs[a:e] = xr
    np.testing.assert_allclose(y, y_ref, rtol=1e-12, atol=1e-12)
    assert np.linalg.norm(xs - x_ref) / np.linalg.norm(x_ref) < 1e-8
