#!/usr/bin/env python
"""Benchmark: FMM-accelerated node-patch matvec throughput (Mnode/s) on one GB300.

Workload: the Kirkwood sphere -- radius 20 A, 64 seeded charges uniform in r < 16 A with
q ~ U(-1, 1), icosphere subdivision 7 (163,842 nodes, 327,680 triangles),
eps_in = 2, eps_out = 80, kappa = 0.104 / A, Chebyshev FMM order 6.  Synthetic input;
the paper's molecules (3K1Q, 1K4R) are not available.

A step is one product y = L x of the discretised operator (Eq. 5): gather, P2M, M2M,
M2L, P2L, L2L, L2P, P2P, near-field correction and assembly, scatter -- the whole
per-iteration hot path of the solver.  Timing: CUDA events on the launching stream
around each product; the L2 cache (129 MB) is flushed by writing a 512 MB buffer
between timed products (outside the events).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload on its
own GPU (the product needs no exchange between GPUs here); value = nodes processed by
all ranks / max-over-ranks time.  --impl reference times the FP64 CPU oracle (dense
direct summation, test infrastructure) on row samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM matvec Mnode/s; solves/s, p50/p99 latency vs plain GPU at <=1e-4 dG error"
UNIT = "Mnode/s"
FLUSH_BYTES = 512 << 20
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def workload(name):
    import synthetic
    if name == "kirkwood":
        return synthetic.kirkwood_sphere()
    if name == "born":
        return synthetic.born_ion()
    if name == "paper_sphere":
        return synthetic.paper_sphere()
    raise SystemExit("unknown workload " + name)


def workload_desc(mol):
    return {"workload": "%s: %d nodes, %d triangles, %d charges, eps %g/%g, kappa %g"
            % (mol.name, mol.n_nodes, mol.n_tris, len(mol.q), mol.eps_in, mol.eps_out, mol.kappa)}


def run_config(mol, args, world, leaf_cap=None):
    return dict(workload_desc(mol), fmm_order=args.order,
                leaf_cap=leaf_cap if leaf_cap else (args.leaf_cap or "library default"),
                precision=["fp32", "mixed: tensor-core M2L"][args.precision],
                l2="flushed between timed products (512 MB write)",
                parallelism="replicas" if world > 1 else "single")


# ------------------------------------------------------------------------------------
# serving: many molecules of uneven size through the continuous-batching server
# ------------------------------------------------------------------------------------
def serving_leg(args):
    """The serving configuration: args.serve_requests solve requests (default 512), each a
    synthetic globule drawn from a seeded pool of args.serve_pool molecules whose atom
    counts are log-uniform in [500, 50,000] (surfaces on a 1.2 A lattice: ~10k-350k nodes),
    with kappa ~ U(0.03, 0.3) drawn per request.  Five arms -- plain FP32 and mixed
    precision, each on 1 and on args.serve_slots server slots, and mixed precision on
    args.serve_slots set-up slots and args.serve_solvers solver threads with batched solves
    (up to args.serve_batch requests of similar size in one lockstep GMRES with fused P2P
    and M2L launches) -- run the same requests:
      * capacity: the first args.serve_burst requests submitted at once (solves/s);
      * latency: all requests on one fixed Poisson arrival trace at 0.9x the capacity of
        plain FP32 on args.serve_slots slots, p50/p99 from submission to result (queueing
        included), solves/s = requests / (last result - first submission).
    Each arm also reports the admitted-memory high-water mark and the largest energy
    difference against the plain FP32 arm on the same slots."""
    import numpy as np

    import paper_1710_06316_gb300 as pb
    import synthetic

    rng = np.random.default_rng(synthetic.SEED_BASE + 3)
    counts = np.exp(rng.uniform(np.log(500), np.log(50000), args.serve_pool)).astype(int)
    t0 = time.perf_counter()
    pool = [synthetic.globule(n_atoms=int(c), index=100 + i, grid=1.2) for i, c in enumerate(counts)]
    t_gen = time.perf_counter() - t0
    reqs = [(int(rng.integers(len(pool))), float(rng.uniform(0.03, 0.3))) for _ in range(args.serve_requests)]
    gaps = rng.exponential(1.0, len(reqs))            # unit-rate gaps, scaled by the rate below

    def run(precision, slots, items, rate=None, batch=1):
        with pb.Server(bytes_budget=int(args.serve_budget_gb * (1 << 30)), max_slots=slots, max_batch=batch,
                       solvers=args.serve_solvers) as srv:
            start = time.perf_counter()
            due = start + np.cumsum(gaps[:len(items)]) / rate if rate else None
            tickets = []
            for k, (i, kap) in enumerate(items):
                if rate:
                    delay = due[k] - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                m = pool[i]
                tickets.append(srv.submit(m.xyz, m.tri, m.atoms, m.q, m.eps_in, m.eps_out, kap,
                                          order=args.order, tol=1e-6, precision=precision,
                                          restart=args.serve_restart, max_restart=5))
            res = [srv.wait(t, 3600) for t in tickets]
            info = srv.info()
        t_first = min(r["t_submit"] for r in res)
        t_last = max(r["t_done"] for r in res)
        bad = [(r["status"], r["error"]) for r in res if r["status"] != "OK"]
        lat = sorted(1e3 * r["latency"] for r in res)
        pq = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
        return {"requests": len(res), "solves_per_s": round(len(res) / (t_last - t_first), 3),
                "p50_ms": round(pq(0.5), 1), "p99_ms": round(pq(0.99), 1),
                "wall_s": round(t_last - t_first, 2), "failed": len(bad), "failures": bad[:3],
                "iters_max": max(r["info"]["iters"] for r in res), "max_running": info["max_running"],
                "reserved_high_water_gb": round(info["bytes_high_water"] / 2**30, 2),
                "used_high_water_gb": round(max(r["bytes_used"] for r in res) / 2**30, 2),
                "slots": slots, "max_batch": batch, "largest_batch": info["max_batch"],
                "mean_batch": round(info["batched_requests"] / info["batches"], 2) if info["batches"] else None,
                }, [r["energy"] for r in res]

    def ediff(e, e_ref):
        return max((abs(a / b - 1) for a, b in zip(e, e_ref) if a and b), default=None)

    fused = "mixed_fused_%dslots" % args.serve_slots
    arms = [("plain_fp32_1slot", 0, 1, 1), ("plain_fp32_%dslots" % args.serve_slots, 0, args.serve_slots, 1),
            ("mixed_1slot", 1, 1, 1), ("mixed_%dslots" % args.serve_slots, 1, args.serve_slots, 1),
            (fused, 1, args.serve_slots, args.serve_batch)]
    burst_items = reqs[:args.serve_burst]
    cap, cap_e = {}, {}
    for name, prec, slots, batch in arms:
        cap[name], cap_e[name] = run(prec, slots, burst_items, batch=batch)
    rate = 0.9 * cap["plain_fp32_%dslots" % args.serve_slots]["solves_per_s"]
    lat, lat_e = {}, {}
    for name, prec, slots, batch in arms:
        lat[name], lat_e[name] = run(prec, slots, reqs, rate=rate, batch=batch)
    out = {}
    for name, prec, slots, batch in arms:
        ref = "plain_fp32_1slot" if slots == 1 else "plain_fp32_%dslots" % args.serve_slots
        out[name] = {"capacity": cap[name], "poisson": lat[name],
                     "energy_max_rel_diff_vs_plain": ediff(lat_e[name], lat_e[ref]),
                     "energy_max_rel_diff_vs_plain_1slot": ediff(lat_e[name], lat_e["plain_fp32_1slot"])}
    mix, pla = "mixed_%dslots" % args.serve_slots, "plain_fp32_%dslots" % args.serve_slots
    return {"workload": "%d requests over a pool of %d synthetic globules (%d-%d nodes), kappa U(0.03, 0.3), "
                        "order %d, GMRES(%d) tol 1e-6, each request = setup + solve + energy" % (
                            len(reqs), len(pool), min(m.n_nodes for m in pool), max(m.n_nodes for m in pool),
                            args.order, args.serve_restart),
            "pool_nodes": [m.n_nodes for m in pool], "pool_atoms": [int(c) for c in counts],
            "pool_generation_s": round(t_gen, 1),
            "arrival_rate_per_s": round(rate, 3),
            "arrival_rule": "Poisson, 0.9 x the burst capacity of plain FP32 on %d slots" % args.serve_slots,
            "capacity_requests": len(burst_items), "arms": out,
            "mixed_vs_plain_same_slots": {
                "capacity_ratio": round(cap[mix]["solves_per_s"] / cap[pla]["solves_per_s"], 3),
                "p50_ratio": round(lat[mix]["p50_ms"] / lat[pla]["p50_ms"], 3),
                "p99_ratio": round(lat[mix]["p99_ms"] / lat[pla]["p99_ms"], 3)},
            "fused_vs_unfused_mixed_same_slots": {
                "capacity_ratio": round(cap[fused]["solves_per_s"] / cap[mix]["solves_per_s"], 3),
                "poisson_solves_per_s_ratio": round(lat[fused]["solves_per_s"] / lat[mix]["solves_per_s"], 3),
                "p50_ratio": round(lat[fused]["p50_ms"] / lat[mix]["p50_ms"], 3),
                "p99_ratio": round(lat[fused]["p99_ms"] / lat[mix]["p99_ms"], 3)}}


# ------------------------------------------------------------------------------------
# globule: FMM order and precision sweep
# ------------------------------------------------------------------------------------
def globule_sweep_leg(args, stream):
    """Synthetic globular protein (2,000-atom compact walk, 0.4 A Gaussian isosurface:
    ~200k nodes, ~400k triangles), FMM order 4 / 6 / 8 in plain FP32 and mixed precision:
    product time (CUDA events, L2 flushed) and the product's relative L2 error against
    the FP64 oracle on 512 sampled rows (smooth x)."""
    import numpy as np
    import torch

    import oracle
    import paper_1710_06316_gb300 as pb
    import synthetic

    mol = synthetic.globule(n_atoms=2000, index=2)
    n = mol.n_nodes
    xh = synthetic.smooth_unknowns(mol.xyz, 3)
    x = torch.tensor(xh.astype(np.float32), device="cuda")
    y = torch.empty_like(x)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    rows = np.sort(np.random.default_rng(5).choice(n, 512, replace=False))
    y1, y2 = oracle.Oracle.for_molecule(mol).matvec_rows(rows, xh)
    ref = np.concatenate([y1, y2])
    out = []
    for order in (4, 6, 8):
        for prec in (0, 1):
            rec = {"order": order, "precision": ["fp32", "mixed"][prec]}
            try:
                h = pb.Handle.for_molecule(mol, order=order, precision=prec, stream=stream.cuda_stream)
            except pb.AfmpbError as e:
                rec["error"] = str(e)[:120]
                out.append(rec)
                continue
            for _ in range(3):
                h.matvec(x, y)
            ev = []
            for i in range(20):
                flush.fill_(float(i))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                h.matvec(x, y)
                b.record(stream)
                ev.append((a, b))
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
            yv = y.cpu().numpy().astype(np.float64)
            got = np.concatenate([yv[rows], yv[n + rows]])
            info = h.info()
            rec.update({"ms_per_product": round(ms, 4), "mnode_per_s": round(n / ms / 1e3, 2),
                        "rel_err_vs_oracle_sampled": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                        "m2l_rank": info["m2l_rank"], "leaf_cap": info["leaf_cap"]})
            h.close()
            out.append(rec)
    return {"workload": "globule: 2000 atoms, %d nodes, %d triangles, eps %g/%g, kappa %g" % (
        n, mol.n_tris, mol.eps_in, mol.eps_out, mol.kappa), "sweep": out}


# ------------------------------------------------------------------------------------
# M2L methods at equal accuracy: dense (compressed) translations against plane waves
# ------------------------------------------------------------------------------------
def m2l_compare_leg(args, mol, stream):
    """The list-2 translations of the headline workload done four ways -- dense compressed
    on the tensor cores (the default), dense compressed in FP32 at the default cutoff and
    at a tighter one, and plane waves (the exponential expansions of FMM97, quadratures
    to 1e-6 of 1/r, FP32) -- each with its product time (CUDA events, L2 flushed), its M2L
    stage time and the product's relative L2 error against the FP64 oracle on 512 sampled
    rows (smooth x).  Equal accuracy is read off the error column."""
    import numpy as np
    import torch

    import oracle
    import paper_1710_06316_gb300 as pb
    import synthetic

    n = mol.n_nodes
    xh = synthetic.smooth_unknowns(mol.xyz, 3)
    x = torch.tensor(xh.astype(np.float32), device="cuda")
    y = torch.empty_like(x)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    rows = np.sort(np.random.default_rng(6).choice(n, 512, replace=False))
    y1, y2 = oracle.Oracle.for_molecule(mol).matvec_rows(rows, xh)
    ref = np.concatenate([y1, y2])
    out = []
    for name, kw in [("dense_tensor_core", dict(precision=1)), ("dense_fp32", dict(precision=0)),
                     ("dense_fp32_tight", dict(precision=0, m2l_tol=1e-7)),
                     ("plane_wave_fp32", dict(precision=0, m2l_method=1))]:
        rec = {"method": name}
        try:
            t0 = time.perf_counter()
            h = pb.Handle.for_molecule(mol, order=args.order, stream=stream.cuda_stream, **kw)
            rec["setup_s"] = round(time.perf_counter() - t0, 3)
        except pb.AfmpbError as e:
            rec["error"] = str(e)[:120]
            out.append(rec)
            continue
        for _ in range(3):
            h.matvec(x, y)
        ev = []
        for i in range(10):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.matvec(x, y)
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
        yv = y.cpu().numpy().astype(np.float64)
        got = np.concatenate([yv[rows], yv[n + rows]])
        prof = h.profile(reps=3, flush=flush, flush_bytes=FLUSH_BYTES)
        st = {k: v for k, v, _ in prof["stages"]}
        m2l = st.get("m2l", 0.0) + st.get("compress", 0.0) + st.get("expand", 0.0)
        info = h.info()
        rec.update({"ms_per_product": round(ms, 4), "m2l_ms": round(m2l, 4),
                    "rel_err_vs_oracle_sampled": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                    "m2l_rank": info["m2l_rank"], "device_gb": round(info["device_bytes"] / 2**30, 2)})
        h.close()
        out.append(rec)
    return {"workload": "%d nodes, order %d; m2l_ms = M2L stage (with the basis changes of the compressed "
                        "forms)" % (n, args.order), "methods": out}


# ------------------------------------------------------------------------------------
# capsid scale: one 10M-node solve
# ------------------------------------------------------------------------------------
def capsid_leg(args, stream):
    """Virus-capsid stand-in: 60 icosahedral copies of a 20,000-atom globule (10,455,600
    nodes, 20,971,440 triangles, 1.2M charges), mixed precision, order 6.  Reports the
    product throughput (CUDA events; the working set is far above L2) and the wall time of
    the whole solve: handle setup (geometry, octree, near field, FMM operators, right-hand
    side by the charge FMM), GMRES to 1e-6, and the energy."""
    import numpy as np
    import torch

    import paper_1710_06316_gb300 as pb
    import synthetic

    t0 = time.perf_counter()
    mol = synthetic.capsid()
    t_gen = time.perf_counter() - t0
    n = mol.n_nodes
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = pb.Handle.for_molecule(mol, order=args.order, tol=1e-6, precision=1, stream=stream.cuda_stream)
    t_setup = time.perf_counter() - t0
    info = h.info()
    x = torch.tensor(synthetic.smooth_unknowns(mol.xyz, 1).astype(np.float32), device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        h.matvec(x, y)
    steps = args.capsid_steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(stream)
        h.matvec(x, y)
        b.record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    prof = h.profile(reps=3)
    peaks, kind = measured_peaks()
    sms = torch.cuda.get_device_properties(x.device).multi_processor_count
    roof_ops, roof = rooflines(prof, info, n, args.order, peaks, kind, 1, sms)
    # end to end through the C ABI with pinned host buffers (H2D + product + D2H)
    xh = x.cpu().pin_memory()
    yh = torch.empty(2 * n, dtype=torch.float32).pin_memory()
    h.matvec_host(xh, yh)
    t0 = time.perf_counter()
    for _ in range(steps):
        h.matvec_host(xh, yh)
    e2e_s = (time.perf_counter() - t0) / steps
    e2e = {"value": round(n / e2e_s / 1e6, 3), "unit": UNIT, "h2d_bytes_per_step": 2 * n * 4,
           "d2h_bytes_per_step": 2 * n * 4, "ms_per_step": round(e2e_s * 1e3, 3)}
    t0 = time.perf_counter()
    f, hh, si = h.solve(raise_on_noconv=False)
    t_solve = time.perf_counter() - t0
    t0 = time.perf_counter()
    energy = h.energy()
    t_energy = time.perf_counter() - t0
    h.close()
    return {"workload": "capsid: %d copies of a %d-atom globule, %d nodes, %d triangles, %d charges, eps %g/%g, "
                        "kappa %g, order %d, mixed precision" % (
                            mol.meta["copies"], mol.meta["n_atoms"] // mol.meta["copies"], n, mol.n_tris,
                            len(mol.q), mol.eps_in, mol.eps_out, mol.kappa, args.order),
            "value": round(n / (ms * 1e-3) / 1e6, 3), "unit": UNIT, "ms_per_product": round(ms, 3),
            "steps": steps, "stages_ms": {a: round(b, 3) for a, b, _ in prof["stages"]},
            "e2e": e2e, "roofline": roof, "rooflines": roof_ops,
            "full_solve_wall_s": round(t_setup + t_solve + t_energy, 3),
            "setup_s": round(t_setup, 3), "gmres_s": round(t_solve, 3), "energy_s": round(t_energy, 3),
            "ms_create": {k: round(v, 1) for k, v in zip(("geometry", "tree", "near", "fmm", "rhs", "graph"),
                                                         info["ms_create"])},
            "iters": si["iters"], "status": si["status"], "res_true": si["res_true"],
            "energy_kcal_mol": energy, "charge_fmm": bool(info["charge_fmm"]),
            "nnz_near": info["nnz_near"], "boxes": info["n_boxes"], "m2l_rank": info["m2l_rank"],
            "device_gb": round(info["device_bytes_peak"] / 2**30, 2), "mesh_generation_s": round(t_gen, 1)}


# ------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + CLOCK_FIELDS, "--format=csv,noheader,nounits",
                 "-i", str(gpu_index), "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------------------------------------
# roofline of the dominant stage
# ------------------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_max_mhz, sms):
    # SMs (read from the device) x 128 FP32 lanes x 2 flop per FMA x max SM clock
    return sms * 128 * 2 * sm_max_mhz * 1e6 / 1e12


# FP32 operations per source-target pair in the P2P kernel (p2p_pair2, one lane of each
# packed operation), counted from its source with an FMA as 2 flop: 44 FP32 arithmetic
# operations (6 adds, 20 multiplies, 18 FMAs) = 62 flop, besides the compare and select of
# the skip test and one rsqrt and one exp2 on the special-function unit.
P2P_FLOP_PER_PAIR = 62


def ncu_traffic(kernel):
    """Per-launch DRAM bytes from the committed ncu summary, if the source files of that
    kernel (listed on its line) are unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(p):
        return None
    import hashlib
    src = os.path.join(ROOT, "paper_1710_06316_gb300", "csrc")
    for line in open(p):
        t = line.split()
        if len(t) >= 4 and not line.startswith("#") and t[0] == kernel:
            h = hashlib.sha1()
            for f in t[3].split(","):
                h.update(open(os.path.join(src, f), "rb").read())
            return float(t[1]) if t[2] == h.hexdigest()[:12] else None
    return None


def rooflines(prof, info, n, order, peaks, kind, precision, sms):
    """One roofline entry per product operator, from the stage times of the live profile
    (CUDA events, L2 flushed, stages serialised): P2P against the FP32 FMA peak (derived:
    SMs x 128 lanes x 2 x max clock), the M2L translations against the measured BF16 peak
    (tensor cores, counting the three split products and the useful one) or the FP32 peak,
    and the near-field SpMV + assembly against the measured HBM copy bandwidth.  Returns
    (entries by stage, the dominant stage's entry)."""
    stages = {name: (ms, launches) for name, ms, launches in prof["stages"]}
    n3 = order ** 3
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32 = fp32_peak_tflops(sm_max, sms)
    fp32_kind = "FP32 FMA, derived: %d SMs (device attribute) x 128 lanes x 2 x %.0f MHz" % (sms, sm_max)
    r = info.get("m2l_rank") or n3                 # compressed translation size, or n^3
    out = {}
    ms, _ = stages["p2p"]
    flop = float(P2P_FLOP_PER_PAIR) * info["n_p2p_pairs"]
    out["p2p"] = {"bound": "alu", "kernel": "k_p2p (packed FP32x2 FMA + MUFU)", "unit": "TFLOP/s",
                  "achieved": flop / (ms * 1e-3) / 1e12, "peak": fp32, "peak_kind": fp32_kind,
                  "peak_source": "derived", "ms_per_launch": ms,
                  "work": "%d pairs x %d flop" % (info["n_p2p_pairs"], P2P_FLOP_PER_PAIR)}
    ms, _ = stages["m2l"]
    if precision == 1:
        flop3 = 3 * 2.0 * r * r * info["n_m2l_pairs"] * 2       # hi*hi, hi*lo, lo*hi; Laplace + Yukawa
        kname = ("k_m2l_ts (target-stationary tcgen05 BF16 x3, FP32 accumulate)" if 0 < r <= 112
                 else "k_m2l_tc (tcgen05 BF16 x3, FP32 accumulate)")
        out["m2l"] = {"bound": "tensor", "kernel": kname,
                      "unit": "TFLOP/s", "achieved": flop3 / (ms * 1e-3) / 1e12, "peak": peaks["bf16_tflops"],
                      "peak_kind": "measured dense BF16 GEMM (burst)", "peak_source": kind,
                      "useful_achieved": flop3 / 3 / (ms * 1e-3) / 1e12, "ms_per_launch": ms,
                      "work": "%d translations x 2 kernels x 3 x 2 r^2 flop, r = %d" % (info["n_m2l_pairs"], r)}
    else:
        flop = 2.0 * r * r * info["n_m2l_pairs"] * 2
        out["m2l"] = {"bound": "alu", "kernel": "k_m2l_c (FP32 FMA)", "unit": "TFLOP/s",
                      "achieved": flop / (ms * 1e-3) / 1e12, "peak": fp32, "peak_kind": fp32_kind,
                      "peak_source": "derived", "ms_per_launch": ms,
                      "work": "%d translations x 2 kernels x 2 r^2 flop, r = %d" % (info["n_m2l_pairs"], r)}
    ms, _ = stages["combine"]
    byts = info["nnz_near"] * 20.0 + n * (8 + 16 + 16 + 8 + 8)
    out["combine"] = {"bound": "hbm", "kernel": "k_combine (near SpMV + Eq. 5 assembly)", "unit": "GB/s",
                      "achieved": byts / (ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                      "peak_kind": "measured copy bandwidth", "peak_source": kind, "ms_per_launch": ms,
                      "work": "%d entries x 20 B + %d nodes x 56 B" % (info["nnz_near"], n)}
    for k, e in out.items():
        e["frac"] = round(e["achieved"] / e["peak"], 4)
        e["achieved"] = round(e["achieved"], 3)
        e["peak"] = round(e["peak"], 3)
        e["ms_per_launch"] = round(e["ms_per_launch"], 5)
        if "useful_achieved" in e:
            e["useful_frac"] = round(e["useful_achieved"] / e["peak"], 4)
            e["useful_achieved"] = round(e["useful_achieved"], 3)
        e["traffic"] = ncu_traffic(k)
    dom = max(out, key=lambda k: out[k]["ms_per_launch"])
    head = dict(out[dom], stage=dom, sms=sms,
                stage_ms={k: round(v[0], 5) for k, v in stages.items()})
    return out, head


def gmres_roofline(sinfo, n, peaks, kind, ms_product):
    """The Krylov side of a solve against HBM: the solve's CUDA-event time minus its
    products' time (each at ms_product, the timed product of the same handle: iters +
    restarts + 1 products), against the bytes its step kernels must move.  Arnoldi step j (one
    fused reduction) reads V_0..V_j and w for the coefficients, V_0..V_j again and w
    (read and written) for the update, w and V_{j+1} for the normalisation, ys / w and
    V_j / xs for the FP32 product's input and output: 16 n (2 j + 8) bytes; a second
    Gram-Schmidt pass adds 16 n (2 j + 6); a cycle's x update 16 n (k + 2).  The time also
    holds the launch gaps and the host wait per cycle, so this is a floor on the fraction."""
    k = int(sinfo["iters"])
    products = k + int(sinfo.get("restarts", 0)) + 1
    ms = float(sinfo["ms_gmres"]) - products * float(ms_product)
    if k <= 0 or ms <= 0:
        return None
    unit = 16.0 * n
    byts = sum(unit * (2 * j + 8) for j in range(k)) + unit * (k + 2)
    byts += int(sinfo.get("second_passes", 0)) * unit * (k + 5)         # at the mean j
    e = {"bound": "hbm", "kernel": "GMRES Arnoldi steps (classical Gram-Schmidt twice: k_gs_first, k_gs_second, "
                                   "k_gs_norm, k_gs_normalize) and the cycle's x update, with the host's waits",
         "unit": "GB/s", "achieved": round(byts / (ms * 1e-3) / 1e9, 3), "peak": round(peaks["hbm_gbs"], 3),
         "peak_kind": "measured copy bandwidth", "peak_source": kind, "ms_per_solve": round(ms, 4),
         "work": "%d Arnoldi steps on %d unknowns: %.1f MB" % (k, 2 * n, byts / 1e6), "traffic": None}
    e["frac"] = round(e["achieved"] / e["peak"], 4)
    return e


# ------------------------------------------------------------------------------------
# oracle timing (CPU)
# ------------------------------------------------------------------------------------
def oracle_rows_rate(mol, rows_target_s=12.0, max_rows=200000):
    """Oracle product rows per second on the host cores: (rows/s, cores, sample text)."""
    import numpy as np

    import oracle
    import synthetic
    o = oracle.Oracle.for_molecule(mol)
    x = synthetic.smooth_unknowns(mol.xyz, 1)
    rng = np.random.default_rng(0)
    rows = rng.choice(mol.n_nodes, 16, replace=False)
    t = time.perf_counter()
    o.matvec_rows(rows, x)
    dt = time.perf_counter() - t
    nrow = int(min(max_rows, max(16, rows_target_s / max(dt / 16, 1e-9))))
    rows = rng.choice(mol.n_nodes, nrow, replace=False)
    t = time.perf_counter()
    o.matvec_rows(rows, x)
    dt = time.perf_counter() - t
    return nrow / dt, oracle.num_threads(), nrow, dt


def oracle_near_rate(mol, seconds=3.0, c_near=2.0):
    """The oracle's near-field setup on the host cores, timed on its own: near-rule
    coefficients (patch quadrature of Eq. 6, self terms included) per second over the
    near sets of randomly sampled rows.  A row's near set is taken by the rule
    |x_p - x_t| < c (rho_p + rho_t) with the oracle's patch radii.  Returns
    (entries/s, rows, entries, seconds)."""
    import numpy as np
    from scipy.spatial import cKDTree

    import oracle
    o = oracle.Oracle.for_molecule(mol, c_near=c_near)
    _, _, rho = o.geometry()
    rng = np.random.default_rng(1)
    kd = cKDTree(mol.xyz)

    def pairs(rows):
        ps, ts = [], []
        cand = kd.query_ball_point(mol.xyz[rows], c_near * (rho[rows] + rho.max()))
        for p, c in zip(rows, cand):
            c = np.asarray(c, np.int64)
            d = np.linalg.norm(mol.xyz[c] - mol.xyz[p], axis=1)
            t = c[d < c_near * (rho[p] + rho[c])]
            ps.append(np.full(t.size, p, np.int64))
            ts.append(t)
        return np.concatenate(ps), np.concatenate(ts)

    p, t = pairs(rng.choice(mol.n_nodes, 8, replace=False))
    t0 = time.perf_counter()
    o.coeffs(p, t, rule=o.NEAR)
    per_row = max((time.perf_counter() - t0) / 8, 1e-6)
    nrow = int(min(mol.n_nodes, max(8, seconds / per_row)))
    p, t = pairs(rng.choice(mol.n_nodes, nrow, replace=False))
    t0 = time.perf_counter()
    o.coeffs(p, t, rule=o.NEAR)
    dt = time.perf_counter() - t0
    return p.size / dt, nrow, int(p.size), dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    import synthetic
    mol = workload(args.workload)
    o = oracle.Oracle.for_molecule(mol)
    x = synthetic.smooth_unknowns(mol.xyz, 1)
    rng = np.random.default_rng(0)
    rows_per_step = args.ref_rows
    for _ in range(args.warmup):
        o.matvec_rows(rng.choice(mol.n_nodes, rows_per_step, replace=False), x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.matvec_rows(rng.choice(mol.n_nodes, rows_per_step, replace=False), x)
    dt = time.perf_counter() - t0
    value = rows_per_step * args.steps / dt / 1e6
    cores = oracle.num_threads()
    sample = ("%d random rows of the %d-node product per step (FP64 direct sum over all %d "
              "sources per row, near rule on the fly); value = rows/s = full-product Mnode/s"
              % (rows_per_step, mol.n_nodes, mol.n_nodes))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": run_config(mol, args, int(os.environ.get("WORLD_SIZE", "1"))), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------
# ------------------------------------------------------------------------------------
# replicas: each rank runs the whole workload on its own GPU (no exchange on the data path)
# ------------------------------------------------------------------------------------
def reduce_max(v, dist=None, device="cpu"):
    """The largest of the ranks' values (the slowest replica sets the job's time)."""
    if dist is None:
        return float(v)
    import torch
    t = torch.tensor([float(v)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world, n_nodes, seconds):
    """Whole-job Mnode/s: every rank processed n_nodes in at most `seconds`."""
    return world * n_nodes / seconds / 1e6


def run_gpu(args):
    import numpy as np
    import torch

    import paper_1710_06316_gb300 as pb
    import synthetic

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    # a real (non-legacy) stream: the library queues all its work on it, so the CUDA
    # events below bracket the product itself
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    mol = workload(args.workload)
    n = mol.n_nodes
    x = torch.tensor(synthetic.smooth_unknowns(mol.xyz, 1).astype(np.float32), device=dev)
    y = torch.empty_like(x)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def max_over_ranks(v):
        return reduce_max(v, dist, dev)

    def timed_products(hh, steps, warmup, sample_clocks=False):
        """Mean product time (ms, CUDA events on the launching stream), L2 flushed."""
        for _ in range(max(warmup, 3)):
            hh.matvec(x, y)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(torch.cuda.current_device()) if sample_clocks else None
        if clocks:
            time.sleep(0.25)
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            hh.matvec(x, y)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks else None
        if dist:
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        return max_over_ranks(sum(ms) / len(ms)), clk

    def solve_latency(hh, reps):
        """Repeated solves (GMRES + energy) on a resident handle: p50 / p99 / solves/s, after
        one untimed solve (it captures the handle's cycle graph)."""
        hh.solve(raise_on_noconv=False)
        lat = []
        out = None
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            f, hv, sinfo = hh.solve(raise_on_noconv=False)
            energy = hh.energy()
            lat.append((time.perf_counter() - t0) * 1e3)
            out = (sinfo, energy)
        lat.sort()
        p = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
        return {"n": reps, "p50_ms": round(p(0.5), 3), "p99_ms": round(p(0.99), 3),
                "solves_per_s": round(1e3 * len(lat) / sum(lat), 3)}, out

    h = pb.Handle.for_molecule(mol, order=args.order, tol=1e-6, leaf_cap=args.leaf_cap,
                               precision=args.precision, stream=stream.cuda_stream)
    info = h.info()
    ms_step, clk = timed_products(h, args.steps, args.warmup, sample_clocks=True)
    value = replica_rate(world, n, ms_step * 1e-3)

    # end to end through the C ABI with pinned host buffers (H2D + product + D2H)
    xh = x.cpu().pin_memory()
    yh = torch.empty(2 * n, dtype=torch.float32).pin_memory()
    for _ in range(3):
        h.matvec_host(xh, yh)
    e2e_steps = max(5, min(args.steps, 200))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        h.matvec_host(xh, yh)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = max_over_ranks(e2e_s)
    e2e = {"value": replica_rate(world, n, e2e_s), "unit": UNIT, "h2d_bytes_per_step": 2 * n * 4,
           "d2h_bytes_per_step": 2 * n * 4, "ms_per_step": e2e_s * 1e3}

    prof = h.profile(reps=5, flush=flush, flush_bytes=FLUSH_BYTES)
    peaks, kind = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof_ops, roof = rooflines(prof, info, n, args.order, peaks, kind, args.precision, sms)

    # solves on the resident handle (outside the timed region): GMRES + energy latency
    lat, (sinfo, energy) = solve_latency(h, args.solve_reps)
    h.close()
    roof_ops["gmres"] = gmres_roofline(sinfo, n, peaks, kind, ms_step)

    # the plain FP32 path (M2L on the CUDA cores) at its own best leaf size, same workload
    plain = None
    if args.precision == 1 and not args.no_plain:
        hp = pb.Handle.for_molecule(mol, order=args.order, tol=1e-6, leaf_cap=args.plain_leaf_cap,
                                    precision=0, stream=stream.cuda_stream)
        ms_p, _ = timed_products(hp, max(5, args.steps // 4), args.warmup)
        lat_p, (sinfo_p, energy_p) = solve_latency(hp, args.solve_reps)
        plain = {"value": round(world * n / (ms_p * 1e-3) / 1e6, 3), "unit": UNIT, "ms_per_step": round(ms_p, 5),
                 "leaf_cap": hp.info()["leaf_cap"], "solve": lat_p, "energy_kcal_mol": energy_p,
                 "energy_rel_diff_vs_mixed": abs(energy_p / energy - 1) if energy else None}
        hp.close()

    line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == 0 else "f32+bf16x3", "data": "synthetic",
            "config": run_config(mol, args, world, info["leaf_cap"]),
            "e2e": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in e2e.items()},
            "roofline": roof,
            "rooflines": roof_ops,
            "gpu_launches": int(prof["kernels_per_product"]) * args.steps,
            "clocks": clk,
            "ms_graph_profile": round(prof["ms_graph"], 5),
            "tree": {"boxes": info["n_boxes"], "leaves": info["n_leaves"], "levels": info["n_levels"],
                     "nnz_near": info["nnz_near"], "p2p_pairs": info["n_p2p_pairs"],
                     "m2l_pairs": info["n_m2l_pairs"], "m2l_rank": info["m2l_rank"],
                     "m2l_tables": info["m2l_tables"], "ms_create": [round(v, 1) for v in info["ms_create"]]},
            "solve": dict(lat, status=sinfo["status"], iters=sinfo["iters"],
                          ms_gmres=round(sinfo["ms_gmres"], 3), ms_products=round(sinfo["ms_matvec_total"], 3),
                          second_passes=sinfo.get("second_passes"), res_true=sinfo["res_true"],
                          energy_kcal_mol=energy),
            "plain_fp32": plain}
    if args.workload == "kirkwood" and energy is not None:
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from closed_forms import kirkwood_energy
        e_ref = kirkwood_energy(mol.atoms, mol.q, mol.meta["radius"], mol.eps_in, mol.eps_out, mol.kappa)
        line["solve"]["kirkwood_series_kcal_mol"] = e_ref
        line["solve"]["energy_rel_err_vs_series"] = abs(energy / e_ref - 1)
    if rank == 0 and world == 1 and not args.no_serving:
        line["serving"] = serving_leg(args)
    if rank == 0 and world == 1 and not args.no_m2l_compare:
        line["m2l_compare"] = m2l_compare_leg(args, mol, stream)
    if rank == 0 and world == 1 and not args.no_sweep:
        line["globule_sweep"] = globule_sweep_leg(args, stream)
    if rank == 0 and world == 1 and not args.no_capsid:
        line["capsid"] = capsid_leg(args, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, nrow, dt = oracle_rows_rate(mol, rows_target_s=args.cpu_seconds)
        line["cpu_baseline"] = {"value": round(rate / 1e6, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "%d random rows of the product in %.1f s (FP64 direct sum, O(N) per "
                                          "row, near rule on the fly); rows/s = full-product Mnode/s" % (nrow, dt)}
        try:
            erate, erows, nent, edt = oracle_near_rate(mol)
            line["cpu_baseline"]["near_setup"] = {
                "entries_per_s": round(erate, 1), "sample": "near sets of %d random rows, %d entries in %.1f s"
                                                            % (erows, nent, edt),
                "full_setup_s_est": round(info["nnz_near"] / erate, 1),
                "gpu_near_setup_ms": round(info["ms_create"][2], 1)}
        except Exception as ex:         # the headline line is printed whatever happens here
            line["cpu_baseline"]["near_setup"] = {"error": repr(ex)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="kirkwood", choices=["kirkwood", "born", "paper_sphere"])
    ap.add_argument("--order", type=int, default=6)
    ap.add_argument("--leaf-cap", type=int, default=0)
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1])
    ap.add_argument("--plain-leaf-cap", type=int, default=0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-pool", type=int, default=16)
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-burst", type=int, default=128)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-batch", type=int, default=8)
    ap.add_argument("--serve-solvers", type=int, default=2)
    ap.add_argument("--serve-budget-gb", type=float, default=96.0)
    ap.add_argument("--serve-restart", type=int, default=80)
    ap.add_argument("--no-capsid", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-m2l-compare", action="store_true")
    ap.add_argument("--capsid-steps", type=int, default=10)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--solve-reps", type=int, default=100)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-rows", type=int, default=48)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
