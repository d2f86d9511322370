#!/usr/bin/env python
"""Benchmark: multi-rhs Wilson-clover Dirac operator and batched GMRES on one GB300.

One "step" is one pass of the whole path over one batch of rhs: upload-free
gauge-field packing (set_gauge from the device copy), clover build and inversion
(set_clover), and an odd-even batched GMRES(32) solve to a 1e-10 true relative
residual with the FP32 operator and Arnoldi process in inner solves of an FP64
iterative refinement (the solve's last step applies the full FP64 operator to
report the final residual).

Workloads (synthetic and seeded: gauge links exp(i eps H) with H a Gaussian su(3) element per
link, Gaussian sources; the generators are in synthetic/):
  solve        16^3 x 32, Wilson-clover c_sw = 1, U = exp(i 0.3 H), m0 = -0.2,
               nrhs = 16 Gaussian sources (the operator-sweep lattice)   [default]
  solve-large  32^3 x 64, U = exp(i 0.25 H), m0 = -0.3, nrhs = 12
  batch, adjoint, apply, ortho: see WORKLOADS below

value = sites x rhs solved per second, summed over ranks (each rank solves its
own batch: weak scaling, no communication). The JSON line also reports the
operator sweep (GB/s against the HBM roofline), the FP64-vs-mixed GMRES
comparison, the roofline of the dominant kernel measured with CUDA events inside
the timed steps, the CPU oracle baseline and an end-to-end number through the
C ABI with host buffers.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the CPU oracle baseline is reported for one host thread
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

METRIC = "multi-rhs Dslash GB/s & site·rhs/s vs HBM roofline; GMRES time-to-1e-10, mixed vs FP64"

WORKLOADS = {
    "solve": dict(name="eo-gmres32-mixed 16^3x32 clover nrhs=16", dims=(32, 16, 16, 16), eps=0.3, m0=-0.2,
                  c_sw=1.0, nrhs=16, gauge_seed=1000, rhs_seed=1001, restart=32, tol=1e-10),
    "solve-large": dict(name="eo-gmres32-mixed 32^3x64 clover nrhs=12", dims=(64, 32, 32, 32), eps=0.25, m0=-0.3,
                        c_sw=1.0, nrhs=12, gauge_seed=2000, rhs_seed=2001, restart=32, tol=1e-10),
    # uneven multi-lattice batch: one step = one lqcd_solve_batch over four lattices of different
    # size, gauge roughness, mass and rhs count (eo GMRES(32), FP32 inner, FP64 refinement, 1e-10)
    "batch": dict(name="uneven batch 8^4/12^4/16^4/16^3x32 nrhs 4/8/16/32 eo-gmres32-mixed", kind="batch",
                  lattices=[((8, 8, 8, 8), 0.2, 0.05, 4), ((12, 12, 12, 12), 0.27, 0.0, 8),
                            ((16, 16, 16, 16), 0.33, -0.05, 16), ((32, 16, 16, 16), 0.4, -0.1, 32)],
                  c_sw=1.0, gauge_seed=3000, rhs_seed=3100, restart=32, tol=1e-10),
    # differentiable solve: one step = forward solve + adjoint solve + link force (the gradient of
    # L = sum_i Re <eta_i, D^{-1} b_i> in b and U)
    "adjoint": dict(name="adjoint eo-gmres32-mixed 16^4 clover nrhs=8 (dL/db, dL/dU)", dims=(16, 16, 16, 16), eps=0.3,
                    m0=-0.05, c_sw=1.0, nrhs=8, gauge_seed=4001, rhs_seed=4002, restart=32, tol=1e-10,
                    kind="adjoint"),
    # single-kernel workloads (one step = one launch group), also the small cases for ncu captures
    "apply": dict(name="schur-apply c64 16^3x32 clover nrhs=16", dims=(32, 16, 16, 16), eps=0.3, m0=-0.2,
                  c_sw=1.0, nrhs=16, gauge_seed=1000, rhs_seed=1001, kind="apply"),
    "ortho": dict(name="cgs2-step c64 16^3x32 odd sites nrhs=16 nvec=16", dims=(32, 16, 16, 16), eps=0.3,
                  m0=-0.2, c_sw=1.0, nrhs=16, gauge_seed=1000, rhs_seed=1001, kind="ortho", nvec=16),
}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) and algorithmic bytes of the
# streaming Gram-Schmidt kernel from one small single-kernel ncu capture (`--workload ortho
# --nvec 32`: the three passes of one 32-vector CGS2 step on the 16^3 x 32 odd sites, 16 rhs;
# the summary is under profiles/). The solve's passes are the same kernel with other flags, so
# the reported traffic per step is the timed solve's algorithmic bytes per step times this
# ratio (FP32 basis; BF16 and other workloads: null).
GS_DRAM_CAPTURE = {("solve", "c64", 2): (3321.959424e6 + 3.148288e6 + 3322.026496e6 + 97.911552e6
                                         + 3321.978624e6 + 97.722624e6,
                                         3 * 3321.888768e6 + 2 * 100.663296e6)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(world, x, device="cuda"):
    """Max over ranks of a host float (the timed region's length)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_rhs_seed(base_seed: int, rank: int) -> int:
    """Each rank solves its own batch of sources (weak scaling over independent rhs)."""
    return base_seed + 7919 * rank


def aggregate_throughput(world: int, units_per_rank_step: float, steps: int, t_max: float) -> float:
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return world * units_per_rank_step * steps / t_max


# ------------------------------------------------------------------ oracle (CPU) arm

def oracle_setup(w):
    """Gauge field, site blocks and one Gaussian rhs of the workload for the FP64 numpy oracle."""
    import oracle
    import synthetic as syn
    U = syn.gauge_field(w["dims"], "exp", w["eps"], seed=w["gauge_seed"])
    b = syn.gaussian_spinors(w["dims"], 1, w["rhs_seed"])
    t0 = time.perf_counter()
    A, Ainv = oracle.diag_blocks(U, w["m0"], w["c_sw"])
    return U, A, Ainv, b, time.perf_counter() - t0


def oracle_cycle(U, A, Ainv, b, m: int):
    """One GMRES(m) cycle of the oracle's odd-even solve on one rhs, as the oracle stands:
    source preparation, the initial residual, m Arnoldi steps, the update, the final
    residual and the reconstruction (m + 2 Schur-operator applies)."""
    import oracle
    t0 = time.perf_counter()
    oracle.solve_eo(U, A, Ainv, b, tol=1e-30, m=m, max_restarts=1)
    return time.perf_counter() - t0


def oracle_apply_sample(w, nrhs: int):
    """The FP64 oracle's Schur and full operator, each applied once to nrhs Gaussian rhs of the
    workload's lattice, timed; returns site*rhs/s of each and the set-up time."""
    import oracle
    import synthetic as syn
    U = syn.gauge_field(w["dims"], "exp", w["eps"], seed=w["gauge_seed"])
    psi = syn.gaussian_spinors(w["dims"], nrhs, w["rhs_seed"] + 17)
    t0 = time.perf_counter()
    A, Ainv = oracle.diag_blocks(U, w["m0"], w["c_sw"])
    t_setup = time.perf_counter() - t0
    C = (4.0 + w["m0"]) * np.eye(12) - A          # C = (4 + m0) - A, no second clover build
    psi_o = oracle.split_parity(psi, 1)
    t0 = time.perf_counter()
    oracle.apply_schur(U, A, Ainv, psi_o)
    t_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.apply_D(U, psi, w["m0"], C)
    t_f = time.perf_counter() - t0
    V = psi.shape[1] * psi.shape[2] * psi.shape[3] * psi.shape[4]
    return {"schur": V // 2 * nrhs / t_s, "full": V * nrhs / t_f, "schur_s": t_s, "full_s": t_f,
            "setup_s": t_setup, "nrhs": nrhs}


_POOL_STATE = {}


def _oracle_pool_init(w):
    """Worker set-up of the all-cores oracle sample: the workload's gauge field and site blocks."""
    import oracle
    import synthetic as syn
    U = syn.gauge_field(w["dims"], "exp", w["eps"], seed=w["gauge_seed"])
    A, Ainv = oracle.diag_blocks(U, w["m0"], w["c_sw"])
    _POOL_STATE.update(U=U, A=A, Ainv=Ainv, dims=w["dims"])


def _oracle_pool_apply(seed):
    import oracle
    import synthetic as syn
    st = _POOL_STATE
    psi_o = oracle.split_parity(syn.gaussian_spinors(st["dims"], 1, seed), 1)
    oracle.apply_schur(st["U"], st["A"], st["Ainv"], psi_o)
    return 1


def oracle_apply_all_cores(w, cores):
    """The oracle's Schur apply on one rhs per host core at once (processes started with spawn): site*rhs/s
    of the whole host, timed over one round of `cores` applies after a warm-up round."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_oracle_pool_init, initargs=(w,)) as pool:
        pool.map(_oracle_pool_apply, range(cores), chunksize=1)
        t0 = time.perf_counter()
        pool.map(_oracle_pool_apply, range(cores, 2 * cores), chunksize=1)
        t = time.perf_counter() - t0
    return V_of(w) // 2 * cores / t, t


def cpu_threads():
    return int(os.environ.get("OPENBLAS_NUM_THREADS", "1"))


def oracle_cost_model(U, A, Ainv, b, m, t_cycle_m):
    """Cost of one Arnoldi step and of the fixed per-cycle work (preparation, residuals, update,
    reconstruction) of the oracle's GMRES: one extra cycle of 2m steps, differenced with the
    measured m-step cycle time."""
    t2m = oracle_cycle(U, A, Ainv, b, 2 * m)
    t_iter = max((t2m - t_cycle_m) / m, 1e-9)
    return t_iter, max(t_cycle_m - m * t_iter, 0.0)


def run_reference(args, w):
    """The oracle arm: per step one GMRES(m) cycle of the oracle's odd-even solve on one rhs of the
    workload (m = --ref-cycle-steps), timed as it stands; ms_per_step is that wall time. value
    projects it to a whole solve in the GPU arm's unit (site*rhs solved per second): the oracle's
    set-up (clover blocks) + the GPU solve's iteration count x the cost of one Arnoldi step + one
    fixed per-cycle cost per GMRES(32) cycle, the step and fixed costs separated by one extra cycle
    of 2m steps timed after the warm-up."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if "dims" not in w:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle arm for the {w['name']} workload; "
                          "the default workload times the oracle"}), flush=True)
        return
    V = w["dims"][0] * w["dims"][1] * w["dims"][2] * w["dims"][3]
    its = args.ref_iterations
    m = args.ref_cycle_steps
    U, A, Ainv, b, t_setup = oracle_setup(w)
    for _ in range(args.warmup):
        oracle_cycle(U, A, Ainv, b, m)
    times = [oracle_cycle(U, A, Ainv, b, m) for _ in range(args.steps)]
    t_step = statistics.mean(times)
    t_iter, t_fixed = oracle_cost_model(U, A, Ainv, b, m, t_step)
    cycles = -(-its // 32)
    t_solve = t_setup + its * t_iter + cycles * t_fixed
    value = V * 1 / t_solve
    sample = (f"per step one oracle GMRES({m}) cycle of the odd-even solve on 1 rhs ({t_step:.2f} s); projected "
              f"to one solve: set-up {t_setup:.1f} s + {its} Arnoldi steps x {t_iter:.2f} s + {cycles} cycles x "
              f"{t_fixed:.2f} s fixed cost ({its} = the GPU solve's iterations per rhs)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "site·rhs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": w["name"]},
            "cpu_baseline": {"value": value, "unit": "site·rhs/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "site·rhs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def op_bytes(V, nrhs, dtype_bytes, op, link_bytes):
    """Algorithmic bytes of one apply: spinors once per pass, each link (link_bytes) and site block
    (72 reals) once per pass. Full: (48 b s + 4 L + 72 s) per site; Schur: (120 b s + 16 L + 144 s)
    per odd site (two passes, each reading all 4V links)."""
    s = dtype_bytes
    if op == "full":
        return V * (48 * nrhs * s + 4 * link_bytes + 72 * s)
    return (V // 2) * (120 * nrhs * s + 16 * link_bytes + 144 * s)


def dslash_point(lat, lq, torch, dims, nrhs, dtype, op, reps, flush):
    V = dims[0] * dims[1] * dims[2] * dims[3]
    sites = lq.SITES_FULL if op == lq.OP_FULL else lq.SITES_ODD
    pin = lat.packed_empty(dtype, sites, nrhs)
    pout = lat.packed_empty(dtype, sites, nrhs)
    g = torch.Generator(device="cuda").manual_seed(nrhs)
    pin.copy_(torch.randn(pin.shape, dtype=pin.dtype, device="cuda", generator=g))
    for _ in range(3):
        lat.apply_packed(op, nrhs, pin, pout)
    s = torch.cuda.current_stream()
    times = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        lat.apply_packed(op, nrhs, pin, pout)
        e1.record(s)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    t = statistics.median(times)
    sz = 8 if dtype == lq.C128 else 4
    if lat.link_storage() == lq.LINKS_BF16 and dtype != lq.C128:
        link_bytes = 12 * 2
    else:
        link_bytes = lat.variant_link_reals(dtype, lat.kernel_variant(dtype, nrhs, op)) * sz
    name = "full" if op == lq.OP_FULL else "schur"
    nbytes = op_bytes(V, nrhs, sz, name, link_bytes)
    units = V * nrhs if op == lq.OP_FULL else (V // 2) * nrhs
    return t, nbytes, units, link_bytes


def run_kernel_workload(args, w):
    """One step = one odd-even Schur apply (c64) or one CGS2 Gram-Schmidt step (c64)."""
    import torch

    world, rank, local = dist_setup()
    from paper_2601_05816_gb300 import _build
    if rank == 0:
        _build.build()
    barrier(world)
    import paper_2601_05816_gb300 as lq
    import synthetic as syn
    lq.load()
    dims, nrhs = w["dims"], w["nrhs"]
    V = dims[0] * dims[1] * dims[2] * dims[3]
    U = syn.gauge_field(dims, "exp", w["eps"], seed=w["gauge_seed"])
    lat = lq.Lattice(dims, time_bc=-1)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(w["m0"], w["c_sw"])
    peak, peak_kind = measured_peaks()
    g = torch.Generator(device="cuda").manual_seed(7 + rank)
    tuning = None
    if w["kind"] == "apply":
        if not (args.no_tune and args.variant >= 0):
            tuning = lat.tune(lq.C64, nrhs, reps=5)
        if args.variant >= 0:
            lat.set_kernel_variant(lq.C64, nrhs, lq.OP_SCHUR, args.variant)
        pin = lat.packed_empty(lq.C64, lq.SITES_ODD, nrhs)
        pin.copy_(torch.randn(pin.shape, dtype=pin.dtype, device="cuda", generator=g))
        pout = torch.empty_like(pin)

        def step():
            lat.apply_packed(lq.OP_SCHUR, nrhs, pin, pout)
        nbytes = (V // 2) * (120 * nrhs + 432) * 4
        launches = 2
        kernel = "dslash_kernel<float,2> (Schur passes A + B)"
    else:
        nvec = w["nvec"]
        n = (V // 2) * 12 * nrhs
        bf16 = args.precision == "bf16"
        if bf16:   # BF16 pairs in 32-bit words
            basis = torch.randint(-2**30, 2**30, (nvec * n,), dtype=torch.int32, device="cuda", generator=g)
            basis &= 0x3f7f3f7f   # finite BF16 values of magnitude < 1
        else:
            basis = torch.randn(nvec * n, dtype=torch.complex64, device="cuda", generator=g)
        wv = torch.randn(n, dtype=torch.complex64, device="cuda", generator=g)
        h = torch.empty((nvec, nrhs), dtype=torch.complex128, device="cuda")
        hn = torch.empty(nrhs, dtype=torch.float64, device="cuda")

        def step():
            lat.orthogonalise(lq.SITES_ODD, nrhs, nvec, basis, wv, h, hn, reorth=True,
                              dtype=lq.BF16S if bf16 else lq.C64)
        vb = 4 if bf16 else 8
        nbytes = 3 * nvec * n * vb + n * 8 * 5
        launches = 7
        kernel = f"gs_stream_kernel ({'BF16' if bf16 else 'FP32'} basis; CGS2 step: dots, update+dots, update+norm)"
    for _ in range(args.warmup):
        step()
    s = torch.cuda.current_stream()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(args.steps):
            step()
        e1.record(s)
        torch.cuda.synchronize()
        barrier(world)
    t_local = e0.elapsed_time(e1) * 1e-3
    t = allreduce_max(world, t_local)
    units = (V // 2) * nrhs
    achieved = nbytes * args.steps / t_local / 1e9
    line = {"metric": METRIC, "value": world * units * args.steps / t, "unit": "site·rhs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": w["name"], "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None,
                         "bytes_per_step": nbytes},
            "clocks": clk.summary(), "gpu_launches": launches * args.steps}
    if tuning is not None:
        line["tuning"] = {"variant_ms_full_schur": tuning,
                          "chosen_schur": lat.kernel_variant(lq.C64, nrhs, lq.OP_SCHUR)}
    lat.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batch_workload(args, w):
    """One step = one lqcd_solve_batch over the workload's lattices; also the same solves one after another."""
    import torch

    world, rank, local = dist_setup()
    from paper_2601_05816_gb300 import _build
    if rank == 0:
        _build.build()
    barrier(world)
    import paper_2601_05816_gb300 as lq
    import synthetic as syn
    lq.load()
    lats, Us, bs, xs, nr, m0s = [], [], [], [], [], []
    units = 0
    for k, (dims, eps, m0, nrhs) in enumerate(w["lattices"]):
        U = torch.from_numpy(syn.gauge_field(dims, "exp", eps, seed=w["gauge_seed"] + k)).cuda()
        b = torch.from_numpy(syn.gaussian_spinors(dims, nrhs, rank_rhs_seed(w["rhs_seed"] + k, rank))).cuda()
        lat = lq.Lattice(dims, time_bc=-1)
        lat.set_gauge(U)
        lat.set_clover(m0, w["c_sw"])
        lat.tune(lq.C64, nrhs, reps=3)
        lat.tune(lq.C128, nrhs, reps=1)
        lats.append(lat); Us.append(U); bs.append(b); xs.append(torch.zeros_like(b)); nr.append(nrhs); m0s.append(m0)
        units += dims[0] * dims[1] * dims[2] * dims[3] * nrhs
    kw = dict(op=lq.OP_SCHUR, precision=lq.C64, restart_len=w["restart"], tol=w["tol"],
              max_restarts=args.max_restarts)
    s = torch.cuda.current_stream()

    def step():
        for x in xs:
            x.zero_()
        return lq.solve_batch(lats, bs, xs, nr, **kw)

    for _ in range(args.warmup):
        step()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(args.steps):
            res = step()
        e1.record(s)
        torch.cuda.synchronize()
        barrier(world)
    t = allreduce_max(world, e0.elapsed_time(e1) * 1e-3)
    for r in res:
        if r.status != lq.OK or r.relres_max > w["tol"]:
            raise SystemExit(f"batch solve did not converge: {r}")
    # the same solves one after another (one lqcd_solve per lattice)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq = []
    for lat, b, x, n in zip(lats, bs, xs, nr):
        x.zero_()
        seq.append(lat.solve(b, x, n, **kw))
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    line = {"metric": METRIC, "value": world * units * args.steps / t, "unit": "site·rhs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp32 inner / fp64 refinement", "data": "synthetic",
            "config": {"workload": w["name"], "lattices": [f"{'x'.join(map(str, d[::-1]))} eps {e} m0 {m} nrhs {n}"
                                                            for d, e, m, n in w["lattices"]]},
            "batch": {"iterations": [r.iterations for r in res], "cycles": [r.restarts for r in res],
                      "fp64_residuals": [r.outer_steps for r in res],
                      "relres_max": [r.relres_max for r in res],
                      "sequential_s": t_seq, "batch_s": t / args.steps,
                      "speedup_vs_sequential": t_seq / (t / args.steps)},
            "clocks": clk.summary()}
    for lat in lats:
        lat.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_adjoint_workload(args, w):
    """One step = x = D^{-1} b (FP32 inner, FP64 refinement), lambda = D^{-dagger} eta, dL/dU (lqcd_force)."""
    import torch

    world, rank, local = dist_setup()
    from paper_2601_05816_gb300 import _build
    if rank == 0:
        _build.build()
    barrier(world)
    import paper_2601_05816_gb300 as lq
    import synthetic as syn
    lq.load()
    dims, nrhs = w["dims"], w["nrhs"]
    V = dims[0] * dims[1] * dims[2] * dims[3]
    U_d = torch.from_numpy(syn.gauge_field(dims, "exp", w["eps"], seed=w["gauge_seed"])).cuda()
    b_d = torch.from_numpy(syn.gaussian_spinors(dims, nrhs, rank_rhs_seed(w["rhs_seed"], rank))).cuda()
    eta_d = torch.from_numpy(syn.gaussian_spinors(dims, nrhs, rank_rhs_seed(w["rhs_seed"], rank) + 1)).cuda()
    lat = lq.Lattice(dims, time_bc=-1)
    kw = dict(op=lq.OP_SCHUR, precision=lq.C64, restart_len=w["restart"], tol=w["tol"],
              max_restarts=args.max_restarts)
    s = torch.cuda.current_stream()

    def step():
        U = U_d.clone().requires_grad_(True)
        b = b_d.clone().requires_grad_(True)
        x = lq.solve_differentiable(lat, U, b, w["m0"], w["c_sw"], **kw)
        (torch.conj(eta_d) * x).real.sum().backward()
        return U.grad, b.grad

    for _ in range(args.warmup):
        step()
    # force kernel alone (the solves dominate the step)
    x = torch.zeros_like(b_d)
    lam = torch.zeros_like(b_d)
    lat.solve(b_d, x, nrhs, **kw)
    lat.solve(eta_d, lam, nrhs, dagger=True, **kw)
    G = torch.empty_like(U_d)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat.force(nrhs, x, lam, G)
    e0.record(s)
    for _ in range(5):
        lat.force(nrhs, x, lam, G)
    e1.record(s)
    torch.cuda.synchronize()
    force_ms = e0.elapsed_time(e1) / 5
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(args.steps):
            gU, gb = step()
        e1.record(s)
        torch.cuda.synchronize()
        barrier(world)
    t = allreduce_max(world, e0.elapsed_time(e1) * 1e-3)
    line = {"metric": METRIC, "value": world * V * nrhs * args.steps / t, "unit": "site·rhs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp32 inner / fp64 refinement; fp64 force", "data": "synthetic",
            "config": {"workload": w["name"], "m0": w["m0"], "c_sw": w["c_sw"],
                       "step": "forward solve + adjoint (gamma5) solve + link force, via torch autograd"},
            "force_kernel_ms": force_ms, "grad_norms": {"dL_dU": float(gU.abs().max()), "dL_db": float(gb.abs().max())},
            "clocks": clk.summary()}
    lat.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_gpu(args, w):
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    from paper_2601_05816_gb300 import _build
    if rank == 0:
        _build.build()
    barrier(world)
    import paper_2601_05816_gb300 as lq
    import synthetic as syn
    lq.load()
    dims, nrhs = w["dims"], w["nrhs"]
    V = dims[0] * dims[1] * dims[2] * dims[3]
    U = syn.gauge_field(dims, "exp", w["eps"], seed=w["gauge_seed"])
    b = syn.gaussian_spinors(dims, nrhs, rank_rhs_seed(w["rhs_seed"], rank))
    U_d = torch.from_numpy(U).cuda()
    b_d = torch.from_numpy(b).cuda()
    x_d = torch.zeros_like(b_d)
    lat = lq.Lattice(dims, time_bc=-1)
    peak, peak_kind = measured_peaks()
    inner = {"c64": lq.C64, "bf16": lq.BF16S}[args.precision]
    solve_kw = dict(op=lq.OP_SCHUR, precision=inner, restart_len=w["restart"], tol=w["tol"],
                    max_restarts=args.max_restarts, use_graph=True, profile=True, reorth=args.reorth)

    # set-up: autotune the hopping kernel for the inner (FP32) and outer (FP64) operators
    lat.set_gauge(U_d)
    lat.set_clover(w["m0"], w["c_sw"])
    tuning = {"c64": lat.tune(lq.C64, nrhs, reps=5), "c128": lat.tune(lq.C128, nrhs, reps=3)}
    if args.variant >= 0:   # e.g. under a profiler, whose serialised launches distort the tuner's timings
        lat.set_kernel_variant(lq.C64, nrhs, lq.OP_SCHUR, args.variant)
    chosen = {k: [lat.kernel_variant(d, nrhs, op) for op in (lq.OP_FULL, lq.OP_SCHUR)]
              for k, d in (("c64", lq.C64), ("c128", lq.C128))}

    def step():
        lat.set_gauge(U_d)
        lat.set_clover(w["m0"], w["c_sw"])
        x_d.zero_()
        return lat.solve(b_d, x_d, nrhs, **solve_kw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    results = []
    s = torch.cuda.current_stream()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(args.steps):
            results.append(step())
        e1.record(s)
        torch.cuda.synchronize()
        barrier(world)
    t_local = e0.elapsed_time(e1) * 1e-3
    t = allreduce_max(world, t_local)
    value = aggregate_throughput(world, V * nrhs, args.steps, t)
    for r in results:
        if r.status != lq.OK or r.relres_max > w["tol"]:
            raise SystemExit(f"solve did not converge: {r}")
    clocks = clk.summary()

    # dominant kernel within the timed steps (profiled with CUDA events on the launching stream)
    op_ms = sum(r.op_ms for r in results)
    gs_ms = sum(r.ortho_ms for r in results)
    if gs_ms >= op_ms:
        ortho = results[0].ortho
        dom = dict(kernel={2: "gs_pass (delayed CGS2 step: 2 streaming passes + coefficient kernels)",
                           1: "gs_pass (CGS2 step: 3 fused passes)"}.get(ortho, "gs_pass (CGS1 step)"),
                   ms=gs_ms, n=sum(r.ortho_launches for r in results),
                   bytes=sum(r.ortho_bytes for r in results),
                   capture=GS_DRAM_CAPTURE.get((args.workload, args.precision, ortho))
                   if "m0_prescribed" not in w else None)
        if dom["capture"] is not None and dom["n"] > 0:
            dram, alg = dom["capture"]
            dom["traffic"] = dom["bytes"] / dom["n"] * dram / alg
        else:
            dom["traffic"] = None
    else:
        dom = dict(kernel="dslash (Schur apply: passes A + B)", ms=op_ms, n=sum(r.op_launches for r in results),
                   bytes=sum(r.op_bytes for r in results), traffic=None)
    achieved = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9 if dom["ms"] > 0 else float("nan")
    roofline = {"bound": "hbm", "kernel": dom["kernel"], "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind, "traffic": dom["traffic"],
                "launches": dom["n"], "avg_launch_ms": dom["ms"] / max(dom["n"], 1),
                "bytes_per_launch": dom["bytes"] / max(dom["n"], 1),
                "share_of_step": (dom["ms"] * 1e-3) / t_local,
                "op_ms": op_ms, "ortho_ms": gs_ms}

    line = {"metric": METRIC, "value": value, "unit": "site·rhs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"c64": "fp32 inner / fp64 refinement",
                      "bf16": "fp32 arithmetic, bf16 Arnoldi basis / fp64 refinement"}[args.precision],
            "data": "synthetic",
            "config": {"workload": w["name"], "lattice": "x".join(str(d) for d in dims[::-1]), "nrhs": nrhs,
                       "gauge": f"exp(i*{w['eps']}*H)", "m0": w["m0"], "c_sw": w["c_sw"],
                       "m0_prescribed": w.get("m0_prescribed", w["m0"]),
                       "solver": f"odd-even GMRES({w['restart']}) FP32 inner solves in FP64 iterative refinement, "
                                 f"tol {w['tol']}",
                       "basis_storage": args.precision,
                       "gram_schmidt": {0: "CGS1", 1: "CGS2", 2: "delayed CGS2"}.get(results[0].ortho, "?"),
                       "parallelism": f"rhs batches, {world} independent rank(s)",
                       "l2": "working set (basis 33 x %.0f MB) far above the 129 MB L2" %
                             ((V // 2) * 12 * nrhs * 8 / 1e6),
                       "timed_path": "profiled solves: CUDA events around every operator and Gram-Schmidt "
                                     "launch, so no graph replay (the graph-replayed solve is gmres.mixed_graph_s)"},
            "roofline": roofline, "clocks": clocks,
            "solve": {"iterations": [r.iterations for r in results], "restarts": [r.restarts for r in results],
                      "fp64_residuals": [r.outer_steps for r in results],
                      "relres_max": max(r.relres_max for r in results),
                      "seconds_host": [r.seconds for r in results]},
            "gpu_launches": int(sum(r.kernel_launches for r in results) + args.steps * 5),
            "tuning": {"variant_ms_full_schur": tuning, "chosen_full_schur": chosen}}

    if rank == 0 and not args.skip_extras:
        extras_sweep(args, w, lat, lq, torch, dims, U_d, peak, line)
        extras_gmres(args, w, lat, lq, torch, b_d, x_d, nrhs, solve_kw, inner, results, line)
        if nrhs <= 16:
            extras_block(args, w, lat, lq, torch, b_d, x_d, nrhs, solve_kw, line)
        extras_e2e(args, w, lat, lq, torch, U, b, nrhs, solve_kw, line)
        extras_oracle_check(args, w, lq, torch, U, b, x_d, lat, nrhs, solve_kw, line)
    lat.close()
    del U_d, b_d, x_d
    torch.cuda.empty_cache()
    if rank == 0 and not args.skip_extras:
        extras_batch(args, lq, torch, line)
        if not args.skip_large:
            extras_gmres_large(args, lq, torch, line)
        # CPU oracle baseline on a bounded sample (rank 0, N = 1 only)
        if world == 1 and not args.skip_cpu:
            extras_cpu_baseline(args, w, line, results)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def extras_sweep(args, w, lat, lq, torch, dims, U_d, peak, line):
    """Operator sweep (dslash GB/s vs the HBM roofline): every nrhs x {c64, c128} x {Schur, full},
    each point the median of --dslash-reps applies with the L2 flushed in between."""
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    lat.set_gauge(U_d)
    lat.set_clover(w["m0"], w["c_sw"])
    # measured SIMT FMA rates: the FP64 applies are bound by them, not by HBM
    alu_peak = {"c64": lq.fma_peak(False), "c128": lq.fma_peak(True)}
    sweep = []
    nr_list = [int(v) for v in args.sweep.split(",")] if args.sweep else [1, 2, 4, 8, 16, 32, 64]
    for nr in nr_list:
        for dt in (lq.C64, lq.C128):
            lat.tune(dt, nr, reps=3)
            for op in (lq.OP_SCHUR, lq.OP_FULL):
                tt, nb, units, lb = dslash_point(lat, lq, torch, dims, nr, dt, op, args.dslash_reps, flush)
                dname = "c64" if dt == lq.C64 else "c128"
                # flops: ~1870 per site and rhs for the full operator (8 x 168 hopping, 504 clover block,
                # scaling and the self term), twice that per odd site and rhs for the Schur complement
                tfl = units * (1870.0 if op == lq.OP_FULL else 3740.0) / tt / 1e12
                sweep.append({"nrhs": nr, "dtype": dname,
                              "op": "schur" if op == lq.OP_SCHUR else "full", "ms": tt * 1e3,
                              "variant": lat.kernel_variant(dt, nr, op), "link_bytes": lb,
                              "GB_s": nb / tt / 1e9, "frac_hbm": nb / tt / 1e9 / peak,
                              "tflops": tfl, "frac_alu": tfl / alu_peak[dname],
                              "site_rhs_per_s": units / tt})
    # BF16 two-row link storage (the FP32 operator with links rounded to BF16) at small rhs counts,
    # where the links are the largest share of the bytes
    bf16_links = []
    lat.set_link_storage(lq.LINKS_BF16)
    for nr in [v for v in nr_list if v <= 8]:
        for op in (lq.OP_SCHUR, lq.OP_FULL):
            tt, nb, units, lb = dslash_point(lat, lq, torch, dims, nr, lq.C64, op, args.dslash_reps, flush)
            ref = next(p for p in sweep if p["nrhs"] == nr and p["dtype"] == "c64" and
                       p["op"] == ("schur" if op == lq.OP_SCHUR else "full"))
            bf16_links.append({"nrhs": nr, "op": "schur" if op == lq.OP_SCHUR else "full", "ms": tt * 1e3,
                               "link_bytes": lb, "GB_s": nb / tt / 1e9, "frac_hbm": nb / tt / 1e9 / peak,
                               "site_rhs_per_s": units / tt, "speedup_vs_fp32_links": ref["ms"] / (tt * 1e3)})
    lat.set_link_storage(lq.LINKS_FP32)
    del flush
    line["dslash"] = {"lattice": line["config"]["lattice"], "bytes_model": "full (48 b s + 4 L + 72 s) per site, "
                      "schur (120 b s + 16 L + 144 s) per odd site; L = bytes per link read (18 or 12 reals)",
                      "l2_flush": "512 MB memset between applies",
                      "applies_per_point": args.dslash_reps, "statistic": "median",
                      "alu_peak_tflops": alu_peak, "alu_peak_kind": "measured (lqcd_fma_peak: SIMT FMA chains)",
                      "points": sweep,
                      "bf16_two_row_links": bf16_links}


def extras_gmres(args, w, lat, lq, torch, b_d, x_d, nrhs, solve_kw, inner, results, line):
    """FP64 plain GPU solve vs the mixed solve of the timed steps (same problem)."""
    lat.set_clover(w["m0"], w["c_sw"])
    torch.cuda.synchronize()
    x_d.zero_()
    t0 = time.perf_counter()
    r64 = lat.solve(b_d, x_d, nrhs, op=lq.OP_SCHUR, precision=lq.C128, restart_len=w["restart"], tol=w["tol"],
                    max_restarts=args.max_restarts, use_graph=True)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    x64 = x_d.clone()
    mixed_s = statistics.mean(r.seconds for r in results)
    x_d.zero_()
    rg = lat.solve(b_d, x_d, nrhs, **dict(solve_kw, profile=False))
    torch.cuda.synchronize()
    diff = [float(torch.linalg.vector_norm(x_d[k] - x64[k]) / torch.linalg.vector_norm(x64[k]))
            for k in range(nrhs)]
    other = {}
    for name, prec in (("c64", lq.C64), ("bf16", lq.BF16S)):
        if prec == inner:
            continue
        x_d.zero_()
        ro = lat.solve(b_d, x_d, nrhs, **dict(solve_kw, precision=prec, profile=False))
        torch.cuda.synchronize()
        other[name] = {"seconds": ro.seconds, "iterations": ro.iterations, "restarts": ro.restarts,
                       "fp64_residuals": ro.outer_steps, "relres": ro.relres_max}
    del x64
    line["gmres"] = {"fp64_s": t64, "mixed_s": mixed_s, "speedup": t64 / mixed_s,
                     "fp64_iterations": r64.iterations, "mixed_iterations": results[-1].iterations,
                     "fp64_relres": r64.relres_max, "mixed_relres": results[-1].relres_max,
                     "mixed_graph_s": rg.seconds, "mixed_vs_fp64_solution_max": max(diff),
                     "other_inner_storage": other,
                     "note": "host wall time of one synchronised solve; mixed_s from the timed steps (profiled, "
                             "no graph replay; mixed_graph_s is the same solve replayed as CUDA graphs)"}


def extras_block(args, w, lat, lq, torch, b_d, x_d, nrhs, solve_kw, line):
    """Block GMRES (one Krylov space for the 16 rhs, FP32 block cycles in FP64 refinement) against the
    batched solver on the same problem: time to solution, Arnoldi steps, true residual."""
    lat.set_clover(w["m0"], w["c_sw"])
    out = {}
    for name, kw in (("batched", dict(solve_kw, profile=False)),
                     ("block", dict(solve_kw, profile=False, block=True, use_graph=False))):
        x_d.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = lat.solve(b_d, x_d, nrhs, **kw)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "status": r.status, "iterations": r.iterations,
                     "fp64_residuals": r.outer_steps, "cycles": r.restarts, "relres_max": r.relres_max}
    out["note"] = ("iterations = Arnoldi steps per rhs; one block step applies the operator to all rhs at once "
                   "and orthogonalises against every rhs's basis vectors")
    line["block_gmres"] = out


def extras_e2e(args, w, lat, lq, torch, U, b, nrhs, solve_kw, line):
    """End to end through the C ABI with pinned host buffers (copies inside the timed region)."""
    U_h = torch.from_numpy(U).pin_memory()
    b_h = torch.from_numpy(b).pin_memory()
    x_h = torch.zeros_like(b_h).pin_memory()
    lat.set_gauge(U_h.numpy())
    lat.set_clover(w["m0"], w["c_sw"])
    lat.solve(b_h.numpy(), x_h.numpy(), nrhs, **dict(solve_kw, profile=False))
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lat.set_gauge(U_h.numpy())
        lat.set_clover(w["m0"], w["c_sw"])
        re = lat.solve(b_h.numpy(), x_h.numpy(), nrhs, **dict(solve_kw, profile=False))
    torch.cuda.synchronize()
    te = (time.perf_counter() - t0) / e2e_steps
    line["e2e"] = {"value": V_of(w) * nrhs / te, "unit": "site·rhs/s", "h2d_bytes_per_step": U.nbytes + b.nbytes,
                   "d2h_bytes_per_step": b.nbytes, "relres_max": re.relres_max,
                   "api": "lqcd_set_gauge + lqcd_set_clover + lqcd_solve with pinned host pointers"}


def V_of(w):
    d = w["dims"]
    return d[0] * d[1] * d[2] * d[3]


def extras_oracle_check(args, w, lq, torch, U, b, x_d, lat, nrhs, solve_kw, line):
    """Per-solve checks against the FP64 oracle: (a) the oracle's residual ||b - D x|| / ||b|| of the
    mixed-precision GPU solution of the timed workload for its first and last rhs; (b) on the 4^4 Haar
    Wilson lattice (m0 = 0.1, GMRES(30)), the error ||x_gpu - x_oracle|| / ||x_oracle|| of the GPU's
    FP64 and mixed solves, full and odd-even, against the oracle's own FP64 GMRES solution."""
    if args.skip_cpu:
        return
    import oracle
    import synthetic as syn
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(w["m0"], w["c_sw"])
    x_d.zero_()
    lat.solve(torch.from_numpy(b).cuda(), x_d, nrhs, **dict(solve_kw, profile=False))
    x = x_d.cpu().numpy()
    sample = [0, nrhs - 1]
    A, _ = oracle.diag_blocks(U, w["m0"], w["c_sw"])
    C = (4.0 + w["m0"]) * np.eye(12) - A
    r = b[sample] - oracle.apply_D(U, x[sample], w["m0"], C)
    rel = [float(np.linalg.norm(r[i]) / np.linalg.norm(b[k])) for i, k in enumerate(sample)]
    small = []
    dims0 = (4, 4, 4, 4)
    U0 = syn.gauge_field(dims0, "haar", seed=0)
    b0 = syn.gaussian_spinors(dims0, 2, 1)
    lat0 = lq.Lattice(dims0, time_bc=-1)
    lat0.set_gauge(U0)
    lat0.set_clover(0.1, 0.0)
    for op, name in ((lq.OP_FULL, "full"), (lq.OP_SCHUR, "eo")):
        if op == lq.OP_FULL:
            xo, _ = oracle.solve_full(U0, None, 0.1, b0, tol=1e-13, m=30, max_restarts=100)
        else:
            A0, Ai0 = oracle.diag_blocks(U0, 0.1, 0.0)
            xo, _ = oracle.solve_eo(U0, A0, Ai0, b0, tol=1e-13, m=30, max_restarts=100)
        for prec, pname in ((lq.C128, "fp64"), (lq.C64, "mixed")):
            xg = np.zeros_like(b0)
            res = lat0.solve(b0, xg, 2, op=op, precision=prec, restart_len=30, tol=1e-10, use_graph=False)
            err = max(float(np.linalg.norm(xg[k] - xo[k]) / np.linalg.norm(xo[k])) for k in range(2))
            small.append({"op": name, "precision": pname, "iterations": res.iterations,
                          "relres_max": res.relres_max, "error_vs_oracle_max": err})
    lat0.close()
    line["oracle_check"] = {
        "timed_workload": {"rhs": sample, "oracle_relres": rel,
                           "note": "the oracle's FP64 operator applied to the GPU's mixed-precision solution"},
        "solution_error_4x4x4x4": {"config": "4^4 Haar Wilson m0 0.1, 2 rhs, GMRES(30) to 1e-10; oracle "
                                             "solution to 1e-13", "solves": small}}


def extras_batch(args, lq, torch, line):
    """The uneven multi-lattice batch (8^4 / 12^4 / 16^4 / 16^3x32 with 4 / 8 / 16 / 32 rhs, one
    lqcd_solve_batch: one captured graph per restart round, a branch per lattice) against the same
    four solves one after another; each the mean of three runs after one warm-up."""
    import synthetic as syn
    wb = WORKLOADS["batch"]
    lats, bs, xs, nr = [], [], [], []
    units = 0
    for k, (dims, eps, m0, nrhs) in enumerate(wb["lattices"]):
        U = torch.from_numpy(syn.gauge_field(dims, "exp", eps, seed=wb["gauge_seed"] + k)).cuda()
        b = torch.from_numpy(syn.gaussian_spinors(dims, nrhs, wb["rhs_seed"] + k)).cuda()
        lat = lq.Lattice(dims, time_bc=-1)
        lat.set_gauge(U)
        lat.set_clover(m0, wb["c_sw"])
        lat.tune(lq.C64, nrhs, reps=3)
        lats.append(lat); bs.append(b); xs.append(torch.zeros_like(b)); nr.append(nrhs)
        units += dims[0] * dims[1] * dims[2] * dims[3] * nrhs
    kw = dict(op=lq.OP_SCHUR, precision=lq.C64, restart_len=wb["restart"], tol=wb["tol"],
              max_restarts=args.max_restarts)

    def batch():
        for x in xs:
            x.zero_()
        return lq.solve_batch(lats, bs, xs, nr, **kw)

    def sequential():
        out = []
        for lat, b, x, n in zip(lats, bs, xs, nr):
            x.zero_()
            out.append(lat.solve(b, x, n, **kw))
        return out

    # each lattice alone: the largest of these bounds any concurrent schedule of the batch from below
    alone = []
    for lat, b, x, n in zip(lats, bs, xs, nr):
        x.zero_()
        lat.solve(b, x, n, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            x.zero_()
            lat.solve(b, x, n, **kw)
        torch.cuda.synchronize()
        alone.append((time.perf_counter() - t0) / 3)
    res = {}
    for name, fn in (("batch", batch), ("sequential", sequential)):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            r = fn()
        torch.cuda.synchronize()
        res[name] = ((time.perf_counter() - t0) / 3, r)
    tb, rb = res["batch"]
    ts, rs_ = res["sequential"]
    line["batch"] = {"workload": wb["name"], "batch_s": tb, "sequential_s": ts, "speedup_vs_sequential": ts / tb,
                     "alone_s": alone, "batch_over_largest_alone": tb / max(alone),
                     "site_rhs_per_s": units / tb, "iterations": [r.iterations for r in rb],
                     "relres_max": [r.relres_max for r in rb],
                     "status": [r.status for r in rb] + [r.status for r in rs_]}
    for lat in lats:
        lat.close()


def extras_gmres_large(args, lq, torch, line):
    """The 32^3 x 64 Wilson-clover workload (eps 0.25, 12 rhs, odd-even GMRES(32) to 1e-10):
    the prescribed mass m0 = -0.3 with the iteration cap --large-cap (status, iterations, true
    residual), then the companion mass --large-m0 where the solve converges: FP32-inner mixed (FP32
    storage, and the BF16 storage variant: BF16 Arnoldi basis and two-row BF16 links) and FP64 plain
    GPU time to solution and their ratios."""
    import synthetic as syn
    wl = WORKLOADS["solve-large"]
    dims, nrhs = wl["dims"], wl["nrhs"]
    t0 = time.perf_counter()
    U = syn.gauge_field(dims, "exp", wl["eps"], seed=wl["gauge_seed"])
    b = syn.gaussian_spinors(dims, nrhs, wl["rhs_seed"])
    t_gen = time.perf_counter() - t0
    U_d = torch.from_numpy(U).cuda()
    b_d = torch.from_numpy(b).cuda()
    del U, b
    x_d = torch.zeros_like(b_d)
    lat = lq.Lattice(dims, time_bc=-1)
    lat.set_gauge(U_d)
    out = {"lattice": "x".join(str(d) for d in dims[::-1]), "nrhs": nrhs, "gauge": f"exp(i*{wl['eps']}*H)",
           "c_sw": wl["c_sw"], "solver": "odd-even GMRES(32), tol 1e-10 (true residual, per rhs)",
           "input_generation_s": t_gen}

    def one(m0, precision, cap, links=lq.LINKS_FP32):
        lat.set_link_storage(links)
        lat.set_clover(m0, wl["c_sw"])
        x_d.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = lat.solve(b_d, x_d, nrhs, op=lq.OP_SCHUR, precision=precision, restart_len=wl["restart"],
                      tol=wl["tol"], max_restarts=cap, use_graph=True)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t
        name = {lq.C64: "fp32 inner / fp64 refinement", lq.BF16S: "fp32 inner arithmetic on bf16-stored basis and "
                "two-row bf16 links / fp64 refinement"}.get(precision, "fp64")
        lat.set_link_storage(lq.LINKS_FP32)
        return {"m0": m0, "precision": name,
                "status": {lq.OK: "converged", lq.NOT_CONVERGED: "not converged"}.get(r.status, str(r.status)),
                "seconds": secs, "iterations": r.iterations, "cycles": r.restarts,
                "fp64_residuals": r.outer_steps, "relres_max": r.relres_max}

    lat.set_clover(wl["m0"], wl["c_sw"])
    lat.tune(lq.C64, nrhs, reps=2)
    lat.tune(lq.C128, nrhs, reps=1)
    out["prescribed"] = one(wl["m0"], lq.C64, args.large_cap)
    out["prescribed"]["note"] = f"capped at {args.large_cap} Arnoldi cycles"
    mixed = one(args.large_m0, lq.C64, args.max_restarts)
    mixed_bf16 = one(args.large_m0, lq.BF16S, args.max_restarts, links=lq.LINKS_BF16)
    fp64 = one(args.large_m0, lq.C128, args.max_restarts)
    out["companion"] = {"m0": args.large_m0, "mixed": mixed, "mixed_bf16_storage": mixed_bf16, "fp64": fp64,
                        "speedup_mixed_vs_fp64": fp64["seconds"] / mixed["seconds"],
                        "speedup_mixed_bf16_storage_vs_fp64": fp64["seconds"] / mixed_bf16["seconds"]}
    lat.close()
    del U_d, b_d, x_d
    torch.cuda.empty_cache()
    line["gmres_large"] = out


def extras_cpu_baseline(args, w, line, results):
    """The oracle as it stands on the host cores: the FP64 Schur and full operator applied once each to
    --cpu-nrhs rhs of the timed workload's lattice (measured, no projection); the projection of the
    oracle's odd-even solve to the GPU solve's iteration count is reported beside it as an extra."""
    smp = oracle_apply_sample(w, args.cpu_nrhs)
    its_gpu = statistics.mean(results[-1].iters_per_rhs)
    U, A, Ainv, b1, t_setup = oracle_setup(w)
    m = args.ref_cycle_steps
    t_cyc = oracle_cycle(U, A, Ainv, b1, m)
    t_iter, t_fixed = oracle_cost_model(U, A, Ainv, b1, m, t_cyc)
    t_proj = t_setup + its_gpu * t_iter + -(-its_gpu // 32) * t_fixed
    all_cores = None
    if args.cpu_all_cores:
        n = os.cpu_count() or 1
        try:
            v_all, t_all = oracle_apply_all_cores(w, n)
            all_cores = {"value": v_all, "unit": "site·rhs/s (FP64 odd-even Schur apply)", "cores": n,
                         "sample": f"{n} processes, one Schur apply on 1 rhs each at once ({t_all:.1f} s)"}
        except Exception as exc:  # e.g. not enough host memory for one oracle per core
            all_cores = {"unavailable": str(exc)[:200]}
    line["cpu_baseline"] = {
        "value": smp["schur"], "unit": "site·rhs/s (FP64 odd-even Schur apply)", "cores": cpu_threads(),
        "all_cores": all_cores,
        "kind": "oracle",
        "sample": f"numpy FP64 oracle on the {w['name'].split(' ')[1]} lattice: one Schur apply and one full "
                  f"apply on {smp['nrhs']} Gaussian rhs, timed ({smp['schur_s']:.1f} s / {smp['full_s']:.1f} s; "
                  f"clover set-up {smp['setup_s']:.1f} s not included)",
        "full_apply_site_rhs_per_s": smp["full"],
        "solve_projection": {"value": V_of(w) / t_proj, "unit": "site·rhs/s (solve, projected)",
                             "method": f"oracle GMRES cycles on 1 rhs: {t_iter:.2f} s per Arnoldi step, {t_fixed:.2f} s "
                                       f"fixed per cycle, scaled to {its_gpu:.0f} iterations + set-up {t_setup:.1f} s"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="solve", choices=sorted(WORKLOADS))
    ap.add_argument("--sweep", default="", help="comma-separated nrhs list for the operator sweep")
    ap.add_argument("--dslash-reps", type=int, default=50)
    ap.add_argument("--skip-extras", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--ref-cycle-steps", type=int, default=2,
                    help="oracle arm: Arnoldi steps of the oracle GMRES cycle timed per step")
    ap.add_argument("--ref-iterations", type=int, default=535,
                    help="oracle arm: iterations per rhs of the GPU solve the oracle's cost is projected to")
    ap.add_argument("--cpu-nrhs", type=int, default=4, help="rhs of the timed oracle operator applies")
    ap.add_argument("--cpu-all-cores", type=int, default=1,
                    help="1: also time the oracle's Schur apply on every host core at once (one process each)")
    ap.add_argument("--skip-large", action="store_true", help="skip the 32^3 x 64 GMRES comparison")
    ap.add_argument("--large-cap", type=int, default=64,
                    help="Arnoldi cycles allowed for the prescribed-mass 32^3 x 64 solve")
    ap.add_argument("--large-m0", type=float, default=-0.1,
                    help="companion mass of the 32^3 x 64 solve (mixed vs FP64 time to solution)")
    ap.add_argument("--m0", type=float, default=None,
                    help="companion run: replace the workload's bare mass (reported as such in config)")
    ap.add_argument("--max-restarts", type=int, default=500)
    ap.add_argument("--precision", default="c64", choices=["c64", "bf16"],
                    help="inner Arnoldi basis storage of the timed solve (FP32 arithmetic either way)")
    ap.add_argument("--nrhs", type=int, default=None,
                    help="apply / ortho workloads: number of rhs (default 16)")
    ap.add_argument("--nvec", type=int, default=None,
                    help="ortho workload: basis size of the timed CGS2 step (default 16)")
    ap.add_argument("--reorth", type=int, default=2, choices=[0, 1, 2],
                    help="solve workloads: Gram-Schmidt of the Arnoldi step (0 CGS1, 1 CGS2, 2 delayed CGS2)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="apply and solve workloads: force this FP32 hopping-kernel launch variant for the Schur "
                         "operator instead of the tuned one")
    ap.add_argument("--no-tune", action="store_true",
                    help="apply workload with --variant: skip the autotuner (only that variant launches)")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.m0 is not None:
        w["m0_prescribed"] = w["m0"]
        w["m0"] = args.m0
        w["name"] += f" (companion run, m0 {args.m0} instead of {w['m0_prescribed']})"
    if args.nrhs is not None and w.get("kind") in ("apply", "ortho"):
        w["name"] = w["name"].replace(f"nrhs={w['nrhs']}", f"nrhs={args.nrhs}")
        w["nrhs"] = args.nrhs
    if args.nvec is not None and w.get("kind") == "ortho":
        w["name"] = w["name"].replace(f"nvec={w['nvec']}", f"nvec={args.nvec}")
        w["nvec"] = args.nvec
    if args.impl == "reference":
        run_reference(args, w)
    elif w.get("kind") in ("apply", "ortho"):
        run_kernel_workload(args, w)
    elif w.get("kind") == "adjoint":
        run_adjoint_workload(args, w)
    elif w.get("kind") == "batch":
        run_batch_workload(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
