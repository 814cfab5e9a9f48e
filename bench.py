#!/usr/bin/env python
"""Benchmark of the cell-wise assembly hot path on GB300.

Workload (default): P2 Lagrange on UnitCubeMesh 64^3 -- 1,572,864 Kuhn tetrahedra, interior vertices
jittered by uniform +-0.2h (seed 0), 129^3 = 2,146,689 dofs -- Helmholtz form, FP64 global CSR.
One step = one pass of every row of the hot path over that mesh:
  sparsity (incidence, per-row sort/unique, CSR, per-cell lookup table) -> zero the Mat ->
  assemble the CSR Mat -> matrix-free action y = A x (x uniform[-1,1], seed 2).
Metric: cells/s (cells of the mesh through one whole step per second).

Multi-GPU: the path shards by mesh (independent problems), so N ranks run N replicas with no
data-path collective (weak scaling); timing is the max over ranks.

--impl reference times the CPU oracle (plain C, FP64) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cells/s assembled (sparsity + CSR assembly + matrix-free action per step)"
METRIC_SERVE = "served Poisson solves/s (assemble + Dirichlet + Jacobi-CG to rtol 1e-8, host to host), p50/p99 latency"
METRIC_BATCH = "cells/s assembled (CSR + RHS of every mesh of the batch per step, sparsity cached)"
WORKLOADS = {
    "p2-3d": dict(dim=3, p=2, n=64, jitter=0.2, seed=0,
                  name="P2 Lagrange UnitCubeMesh 64^3 (1,572,864 Kuhn tets, +-0.2h jitter seed 0, 2,146,689 dofs), "
                       "Helmholtz, FP64 CSR: sparsity + assembly + matrix-free action"),
    "p1-2d": dict(dim=2, p=1, n=64, jitter=0.0, seed=0,
                  name="P1 Lagrange UnitSquareMesh 64x64 (8192 cells, 4225 nodes), Helmholtz, FP64 CSR: "
                       "sparsity + assembly + matrix-free action"),
    "p1-sweep": dict(sweep=True, dim=2, p=1, ns=[256, 512, 1024, 2048], jitter=0.0, seed=0,
                     name="P1 Lagrange UnitSquareMesh n x n for n = 256..2048 (up to 8,388,608 cells), Helmholtz, "
                          "FP64 CSR: assembly roofline sweep (labelled extra; sparsity built once per n)"),
    "wave": dict(wave=True, dim=3, p=1, n=64, jitter=0.2, seed=0, dt=0.001,
                 name="explicit linear wave (lumped mass, Sec. 6.3) on P1 UnitCubeMesh 64^3 (1,572,864 Kuhn tets, "
                      "+-0.2h jitter seed 0, 274,625 nodes), p = sin(10 pi t) on y = 0, dt = 0.001: one time step = "
                      "pull action element kernel + fused per-node update"),
    "p4-kappa": dict(p4=True, dim=2, p=4, n=512, jitter=0.0, seed=0, kappa_seed=3,
                     name="P4 Lagrange UnitSquareMesh 512x512 (524,288 triangles, 4,198,401 dofs), kappa-diffusion "
                          "kappa*inner(grad u, grad v) dx with kappa = exp(N(0,1)) per P1 node (seed 3): zero + CSR "
                          "assembly with element tensors on the tensor cores (three TF32 products), FP64 CSR"),
    "cg": dict(cg=True, name="Jacobi-CG iteration of the largest serving request alone"),
    "batch": dict(count=2048, seed=4, lo=8, hi=256,
                  name="2048 UnitSquareMesh n x n meshes, n log-uniform in [8,256] (seed 4), each P1 or P2 "
                       "(Bernoulli 1/2), Helmholtz CSR + RHS f v dx (f uniform[-1,1] per node, seed 1000+i), "
                       "one persistent launch under a CUDA graph, tuned tile and grid"),
    "serve": dict(serve=True, count=64, seed=5, lo=16, hi=512, budget=2 << 30, max_active=64, tick=16,
                  name="Poisson solve requests on UnitSquareMesh n x n, n log-uniform in [16,512] (seed 5), P1 or P2, "
                       "f from u = sin(k pi x) sin(m pi y), k, m uniform in 1..4, u = 0 on the boundary; pull assembly, "
                       "Dirichlet elimination, Jacobi-CG rtol 1e-8 (FP64 dots); Poisson arrivals, admission by a "
                       "2 GiB device-memory budget"),
}
# ncu dram bytes (read + write) per launch of the dominant kernel, with the sha1 of the kernel
# source they were taken from and what ncu showed binds it; reported as null once the source has
# changed.
TRAFFIC = {
    # k_mat_push<3,2,HELMHOLTZ,f32x2>: 249.0 MB at 40^3 (384,000 cells), scaled x4.096 to 64^3
    ("assemble", "push", "f32x2"): (1.020e9, "c827e6c081c1",
                                    "FP64 atomics in L2 (ncu at 40^3: L2 throughput 50%, 24% warps active)"),
    # the fused phase: the Mat zero (54.7 MB written at 40^3) and k_mat_action_push<3,2,HELMHOLTZ,FP64>
    # (193.9 MB read, 76.8 MB written at 40^3), 325.4 MB, scaled x4.096 to 64^3
    ("assemble_action", "push", "fp64"): (1.333e9, "47eb134234aa",
                                          "FP64 pipe 76% busy beside FP64 reductions in L2 (ncu at 40^3: L2 58%, "
                                          "23.4% warps active at 128 registers, table staged in shared memory)"),
    # one sparsity rebuild (zero, the guarded k_inc_fill, the in-place k_rows_build pass and the gated
    # launches that return at once; column tracking off): 117.3 MB at 40^3, scaled x4.096 to 64^3
    ("sparsity", None, None): (0.4804e9, "f848f281fef1",
                               "integer instruction issue (ncu at 40^3, row pass: issue active 64%, ALU pipe 65%, "
                               "314 warp instructions per row)"),
}


def _src_hash(name):
    p = os.path.join(ROOT, "paper_1501_01809_gb300", "csrc", name)
    with open(p, "rb") as fh:
        return hashlib.sha1(fh.read()).hexdigest()[:12]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 peak: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (nominal GB300 figure 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


class _NvmlSampler:
    """SM clock and clock-event reasons read through NVML (ctypes) by a thread every few
    milliseconds, so that even a timed region of tens of milliseconds gets tens of samples.
    Read-only: it changes no setting of the GPU."""
    # nvmlClocksEventReason bits
    BITS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown", 0x4: "sw_power_cap"}

    def __init__(self, device_index, period_s=0.005):
        import ctypes
        import threading
        self.ct, self.period = ctypes, period_s
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        rc = -1
        try:
            import torch
            pr = torch.cuda.get_device_properties(device_index)
            bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0".encode()
            rc = self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(self.h))
        except Exception:
            rc = -1
        if rc != 0 and self.lib.nvmlDeviceGetHandleByIndex_v2(device_index, ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        self.max_mhz = float(mx.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0 else None
        self.samples, self.stop = [], threading.Event()
        self.thread = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        ct = self.ct
        clk, rs = ct.c_uint(), ct.c_ulonglong()
        while not self.stop.is_set():
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(clk)) == 0 and \
                    self.reasons_fn(self.h, ct.byref(rs)) == 0:
                self.samples.append((float(clk.value), int(rs.value)))
            self.stop.wait(self.period)

    def start(self):
        self.thread.start()

    def finish(self):
        self.stop.set()
        self.thread.join(timeout=2)
        sm = [c for c, _ in self.samples]
        reasons = sorted({name for _, r in self.samples for bit, name in self.BITS.items() if r & bit})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
                "sm_mhz_min": min(sm) if sm else None, "reasons": reasons, "samples": len(sm),
                "source": f"NVML every {self.period * 1e3:.0f} ms during the timed region"}


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"fe_clocks_{os.getpid()}.csv")

    def __enter__(self):
        self.nvml = None
        try:
            self.nvml = _NvmlSampler(self.dev)
            self.nvml.start()
            return self
        except Exception:
            self.nvml = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.nvml is not None:
            self.result = self.nvml.finish()
            return
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.nvml is not None:
            return self.result
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "source": "nvidia-smi every 100 ms"}


# --------------------------------------------------------------------------------------- ranks

def max_over_ranks(x, device=None):
    """Maximum of x over the ranks of the default process group (x itself when not distributed).
    Replicas exchange nothing else: this is the only collective of a multi-rank run."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device if device is not None else "cpu")
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def bind_to_gpu_cpus(dev_index):
    """Restrict this process to the CPUs local to the GPU (sysfs local_cpulist of its PCI function),
    so that pinned host buffers are allocated on the GPU's own socket and host copies do not cross
    the link between sockets.  Returns the CPU list, or None where sysfs does not say (no change)."""
    import torch
    try:
        pr = torch.cuda.get_device_properties(dev_index)
        addr = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{addr}/local_cpulist") as fh:
            spec = fh.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                lo, hi = part.split("-")
                cpus.update(range(int(lo), int(hi) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return f"{addr}: CPUs {spec}"
    except Exception:  # no sysfs entry, no PCI fields, no permission: leave the affinity alone
        return None


def job_throughput(units_per_rank, world, ms_max):
    """Whole-job rate: every rank processes units_per_rank in at most ms_max milliseconds."""
    return world * units_per_rank / (ms_max / 1e3)


# --------------------------------------------------------------------------------------- workload

def make_inputs(wl):
    from paper_1501_01809_gb300 import meshgen as mg
    mesh = (mg.unit_square_mesh if wl["dim"] == 2 else mg.unit_cube_mesh)(wl["n"], wl["jitter"], wl["seed"])
    cmap, nn = mg.cell_node_map(mesh, wl["p"])
    x = mg.uniform_dat(nn, 2)
    return mesh, cmap, nn, x


def counts_per_cell(dim, p):
    """FP64 work per cell of the assembly and action kernels, in FMA-equivalent flops (2 per FP64
    instruction, so that the fraction of the FP64 peak is the FP64 pipe's utilisation): the
    geometry (about 70 FP64 instructions on a tetrahedron, 25 on a triangle), the generated
    Helmholtz element entries after the generator's rewriting (shared pair sums, one product per
    distinct mass value) and, for the action, ND^2 multiply-adds for y = K x."""
    from paper_1501_01809_gb300 import codegen
    nd = len(codegen.lattice_nodes(dim, p))
    temps, reduced = codegen.cse_plan(codegen.stiffness_forms(dim, p))
    elem = len(temps) + sum(len(t) for t in reduced) + len(codegen.mass_values(dim, p))
    geo = 70 if dim == 3 else 25
    return nd, 2 * (geo + elem), 2 * (geo + elem + nd * nd)


def run_ours(args, wl, rank, world):
    import torch
    from paper_1501_01809_gb300 import build as fb
    from paper_1501_01809_gb300 import fe

    fb.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    mesh, cmap, nn, x = make_inputs(wl)
    stream = torch.cuda.Stream(dev)
    ctx = fe.ctx_create(dev.index, stream=stream)
    t_map = torch.from_numpy(cmap).to(dev)
    t_cv = torch.from_numpy(mesh.cell_vertex).to(dev)
    t_xy = torch.from_numpy(mesh.coords).to(dev)
    t_x = torch.from_numpy(x).to(dev)
    t_y = torch.zeros_like(t_x)
    cells, nodes, verts = fe.set_create(ctx, mesh.ncell), fe.set_create(ctx, nn), fe.set_create(ctx, mesh.nvert)
    M = fe.map_create(ctx, cells, nodes, t_map, validate=True)
    CM = fe.map_create(ctx, cells, verts, t_cv, validate=True)
    XY = fe.dat_create(ctx, verts, t_xy)
    X, Y = fe.dat_create(ctx, nodes, t_x), fe.dat_create(ctx, nodes, t_y)
    strat = {"push": fe.STRATEGY_PUSH, "pull": fe.STRATEGY_PULL, "auto": fe.STRATEGY_AUTO}[args.strategy]
    prec = {"fp64": fe.PREC_FP64, "f32x2": fe.PREC_F32X2}[args.precision]
    K = fe.kernel_create(ctx, fe.FORM_HELMHOLTZ, wl["dim"], wl["p"], precision=prec, strategy=strat)
    kcur = [K]  # the kernel the step uses (the labelled double-float extra swaps it)
    with torch.cuda.stream(stream):
        sp = fe.sparsity_build(ctx, M, M)
        A = fe.mat_create(ctx, sp)
    nrows, ncols, nnz, rowptr, colidx = fe.sparsity_csr(sp)
    vals = fe.mat_values(A)

    pull = args.strategy in ("pull", "auto")
    # The Mat zero and the push action depend on neither the rebuilt pattern nor the assembly, so with
    # --overlap they run on a second stream, concurrently with the sparsity rebuild (the pull action
    # reads the rebuilt incidence and stays on the main stream).
    side = None
    if args.overlap != "off" and not pull:
        side = torch.cuda.Stream(dev, priority=-1 if args.overlap in ("hi", "asm-hi") else 0)
    beside_asm = args.overlap in ("asm", "asm-hi")  # the action beside the assembly, after the rebuild
    # --fuse on (FP64 push on one stream): the Mat zero, assembly and action as one call,
    # fe_assemble_mat_action, each cell's element matrix built once for both outputs; fuse[0] is
    # switched off while the double-float extra runs (its separate kernels are the faster ones)
    fuse = [args.fuse == "on" and not pull and side is None and args.precision == "fp64"]

    def compute(sp_, A_, X_, Y_, M_, XY_, CM_, ev=None, sev=None):
        """One pass of the hot path: sparsity rebuild, Mat zero, assembly, action.  ev: 5 events on the
        main stream (start, after the rebuild, before the assembly, after it, end); sev: 2 events on the
        side stream (after the zero, after the action)."""
        if ev is not None:
            ev[0].record(stream)
        if side is None and fuse[0]:  # phases: rebuild | (zero, in the fused call) | fused | (action, in it)
            fe.sparsity_rebuild(sp_)
            if ev is not None:
                ev[1].record(stream)
                ev[2].record(stream)
            fe.assemble_mat_action(ctx, kcur[0], cells, A_, X_, Y_, M_, XY_, CM_, zero_first=True)
            if ev is not None:
                ev[3].record(stream)
                ev[4].record(stream)
            return
        if side is None:
            fe.sparsity_rebuild(sp_)
            if ev is not None:
                ev[1].record(stream)
            if not pull:  # the pull row owners overwrite (zero_first) instead: no separate zero pass
                fe.mat_zero(A_)
            if ev is not None:
                ev[2].record(stream)
            fe.assemble_mat(ctx, kcur[0], cells, A_, XY_, CM_, zero_first=pull)
            if ev is not None:
                ev[3].record(stream)
            fe.action(ctx, kcur[0], cells, X_, Y_, M_, XY_, CM_, zero_first=True, sp=sp_)
            if ev is not None:
                ev[4].record(stream)
            return
        if beside_asm:  # rebuild; then zero + assembly on the main stream, the action beside them
            e1 = ev[1] if ev is not None else torch.cuda.Event()
            ea = sev[1] if sev is not None else torch.cuda.Event()
            fe.sparsity_rebuild(sp_)
            e1.record(stream)
            side.wait_event(e1)
            if sev is not None:
                sev[0].record(side)
            fe.ctx_set_stream(ctx, side)
            try:
                fe.action(ctx, kcur[0], cells, X_, Y_, M_, XY_, CM_, zero_first=True, sp=sp_)
                ea.record(side)
            finally:
                fe.ctx_set_stream(ctx, stream)
            fe.mat_zero(A_)
            if ev is not None:
                ev[2].record(stream)
            fe.assemble_mat(ctx, kcur[0], cells, A_, XY_, CM_, zero_first=False)
            if ev is not None:
                ev[3].record(stream)
            stream.wait_event(ea)
            if ev is not None:
                ev[4].record(stream)
            return
        e0 = ev[0] if ev is not None else torch.cuda.Event()
        if ev is None:
            e0.record(stream)
        ez = sev[0] if sev is not None else torch.cuda.Event()
        ea = sev[1] if sev is not None else torch.cuda.Event()
        side.wait_event(e0)
        fe.ctx_set_stream(ctx, side)
        try:
            fe.mat_zero(A_)
            ez.record(side)
            fe.action(ctx, K, cells, X_, Y_, M_, XY_, CM_, zero_first=True, sp=sp_)
            ea.record(side)
        finally:
            fe.ctx_set_stream(ctx, stream)
        fe.sparsity_rebuild(sp_)
        if ev is not None:
            ev[1].record(stream)
        stream.wait_event(ez)
        if ev is not None:
            ev[2].record(stream)
        fe.assemble_mat(ctx, K, cells, A_, XY_, CM_, zero_first=False)
        if ev is not None:
            ev[3].record(stream)
        stream.wait_event(ea)
        if ev is not None:
            ev[4].record(stream)

    def step(ev=None, sev=None):
        compute(sp, A, X, Y, M, XY, CM, ev, sev)

    for _ in range(args.warmup):
        step()
    fe.sync(ctx)
    # --graph: the whole step (rebuild, zero, assembly, action) captured once as a CUDA graph and
    # replayed, so the launch latency of its 17 kernels is paid once per graph instead of per kernel
    graph = None
    use_graph = args.graph == "on" or (args.graph == "auto" and not pull)
    if use_graph:
        if pull:
            raise SystemExit("--graph on: the push strategy only")
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream, capture_error_mode="thread_local"):
            step()
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                graph.replay()
        fe.sync(ctx)
    dist = world > 1
    if dist:
        import torch.distributed as td
        td.barrier()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    sevs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    # Workloads that fit in L2 (the 8192-cell P1 case) overwrite a 256 MB buffer between steps, outside
    # the timed intervals, so every step starts cold; the large ones have inputs beyond L2.
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if mesh.ncell < 200_000 else None

    def flush_l2():
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.fill_(1)

    with ClockSampler(dev.index) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush_l2()
            step(evs[k], sevs[k])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if dist:
        td.barrier()
    fe.sync(ctx)
    def phase_sums(evs_, sevs_):
        out = np.zeros(4)
        for ev, sev in zip(evs_, sevs_):
            if side is None:
                for q in range(4):
                    out[q] += ev[q].elapsed_time(ev[q + 1])
            elif beside_asm:  # zero and assembly on the main stream, the action beside them
                out += [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3]),
                        sev[0].elapsed_time(sev[1])]
            else:  # live durations of the concurrent phases (sparsity on the main stream, zero and action beside it)
                out += [ev[0].elapsed_time(ev[1]), ev[0].elapsed_time(sev[0]), ev[2].elapsed_time(ev[3]),
                        sev[0].elapsed_time(sev[1])]
        return out

    phases = phase_sums(evs, sevs)
    per_step = sorted(ev[0].elapsed_time(ev[4]) for ev in evs)
    # back to back, the span of all steps; with flushes in between, the sum of the steps
    total_ms = evs[0][0].elapsed_time(evs[-1][4]) if flush is None else sum(per_step)
    ms_step = total_ms / args.steps
    step_stats = {"min_ms": per_step[0], "median_ms": per_step[len(per_step) // 2], "max_ms": per_step[-1]}
    if graph is not None:  # the step time of record is the graph's; the phases above come from launches
        step_stats["eager_ms"] = ms_step
        gev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
        if dist:
            td.barrier()
        torch.cuda.synchronize()
        with ClockSampler(dev.index) as clk:
            t0 = time.perf_counter()
            for k in range(args.steps):
                flush_l2()
                with torch.cuda.stream(stream):
                    gev[k][0].record(stream)
                    graph.replay()
                    gev[k][1].record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        fe.sync(ctx)
        per_step = sorted(a.elapsed_time(b) for a, b in gev)
        ms_step = (gev[0][0].elapsed_time(gev[-1][1]) if flush is None else sum(per_step)) / args.steps
        step_stats.update({"min_ms": per_step[0], "median_ms": per_step[len(per_step) // 2], "max_ms": per_step[-1]})
    if dist:
        ms_step = max_over_ranks(ms_step, dev)
    phase_ms = phases / args.steps

    # ------------------------------------------------------------------- labelled extra: double-float
    # The same step with element tensors in FP32 pairs (double-float, about 2^-46 relative per
    # operation) and FP64 global accumulation: a narrower arithmetic than the FP64 step of record,
    # reported beside it with its own dtype, never as the headline.
    f32x2 = None
    if args.precision == "fp64" and graph is not None and not args.no_f32x2:
        K32 = fe.kernel_create(ctx, fe.FORM_HELMHOLTZ, wl["dim"], wl["p"], precision=fe.PREC_F32X2, strategy=strat)
        kcur[0] = K32
        fused_main, fuse[0] = fuse[0], False
        for _ in range(args.warmup):
            step()
        fe.sync(ctx)
        torch.cuda.synchronize()
        ph32 = np.zeros(4)
        for k in range(args.steps):
            flush_l2()
            step(evs[k], sevs[k])
        torch.cuda.synchronize()
        ph32 = phase_sums(evs, sevs)
        g32 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g32, stream=stream, capture_error_mode="thread_local"):
            step()
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                g32.replay()
        fe.sync(ctx)
        torch.cuda.synchronize()
        gev32 = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
        for k in range(args.steps):
            flush_l2()
            with torch.cuda.stream(stream):
                gev32[k][0].record(stream)
                g32.replay()
                gev32[k][1].record(stream)
        torch.cuda.synchronize()
        fe.sync(ctx)
        ms32 = (gev32[0][0].elapsed_time(gev32[-1][1]) if flush is None else
                sum(a.elapsed_time(b) for a, b in gev32)) / args.steps
        if dist:
            ms32 = max_over_ranks(ms32, dev)
        ph32 /= args.steps
        f32x2 = {"value": job_throughput(mesh.ncell, world, ms32), "unit": "cells/s", "ms_per_step": ms32,
                 "dtype": "f32x2 element / f64 accumulate",
                 "precision": "element tensors in FP32 pairs (double-float, about 2^-46 relative), FP64 CSR and y",
                 "phases_ms": {"sparsity": ph32[0], "zero": ph32[1], "assemble": ph32[2], "action": ph32[3]},
                 "schedule": "serial on one stream, assembly and action as separate kernels (faster in double-float)",
                 "note": "labelled extra, not the step of record: same step and graph schedule, narrower element "
                         "arithmetic"}
        kcur[0] = K
        fuse[0] = fused_main
        del g32
        # the step of record leaves A and y in FP64: restore them for the checks below
        step()
        fe.sync(ctx)
    # launches of libfe kernels per step: sparsity rebuild 13 (zero, count, scan x3, zero, fill, in-place
    # row pass, then the gated full row pass, scan x3 and compact, which return at once when no row
    # changed length); push: mat zero 1, assembly 1, action zero + action 2, or fused: the two zeros
    # and the fused kernel 3; pull: assembly 2 (element, row), action 2 (element, row)
    launches = (13 + (3 if fuse[0] else 4)) * args.steps

    # ------------------------------------------------------------------- e2e through host buffers
    # Every step copies its inputs (maps, coordinates, x) from pinned host memory and its outputs
    # back (CSR values and y; rowptr and colidx when the step's rebuild changed them).  The copies of
    # neighbouring steps overlap the compute on separate streams: three device slots of inputs and
    # outputs, ordered by events.  Each direction's bytes are cut into --copy-streams pieces of about
    # equal size, each on its own stream, so that more than one copy engine can serve a direction.
    e2e = None
    if not args.no_e2e:
        host_cpus = bind_to_gpu_cpus(dev.index)  # pinned buffers on the GPU's own socket
        ncs = max(1, args.copy_streams)
        pin = lambda t: torch.empty(t.shape, dtype=t.dtype, pin_memory=True).copy_(t.cpu())
        host_in = [pin(t) for t in (t_map, t_cv, t_xy, t_x)]
        # Three device slots.  Every step reads back the Mat values, y and the rebuild's two flags; the
        # pattern (rowptr, colidx) is read back only after a rebuild that reports a change
        # (fe_sparsity_changed, with column tracking on: the in-place row pass compares each column
        # it writes), so the host always holds the current pattern.  A slot's flags are checked when
        # the slot comes round again, three steps later, before its next rebuild.
        nslots = 3
        slots = []
        for sidx in range(nslots):
            d_in = [torch.empty_like(t) for t in (t_map, t_cv, t_xy, t_x)]
            for d, h in zip(d_in, host_in):
                d.copy_(h)
            d_y = torch.zeros_like(t_x)
            torch.cuda.synchronize()  # the slot's inputs are on the device before the library reads them
            with torch.cuda.stream(stream):
                Ms = fe.map_create(ctx, cells, nodes, d_in[0])
                CMs = fe.map_create(ctx, cells, verts, d_in[1])
                XYs = fe.dat_create(ctx, verts, d_in[2])
                Xs, Ys = fe.dat_create(ctx, nodes, d_in[3]), fe.dat_create(ctx, nodes, d_y)
                sps = fe.sparsity_build(ctx, Ms, Ms)
                fe.sparsity_track_columns(sps, True)  # exact flags: the rebuild compares what it writes
                As = fe.mat_create(ctx, sps)
            fe.sync(ctx)
            _, _, _, rps, cis = fe.sparsity_csr(sps)
            outs = [fe.mat_values(As), d_y, fe.sparsity_changed(sps)]
            h_out = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in outs]
            pat = [rps, cis]
            h_pat = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True).copy_(t) for t in pat]  # set-up read
            ev = {"in": [torch.cuda.Event() for _ in range(ncs)], "comp": torch.cuda.Event(),
                  "out": [torch.cuda.Event() for _ in range(ncs)]}
            slots.append(dict(d_in=d_in, M=Ms, CM=CMs, XY=XYs, X=Xs, Y=Ys, sp=sps, A=As, outs=outs, h_out=h_out,
                              pat=pat, h_pat=h_pat, ev=ev, used=False))
        s_in = [torch.cuda.Stream(dev) for _ in range(ncs)]
        s_out = [torch.cuda.Stream(dev) for _ in range(ncs)]
        h2d = sum(h.numel() * h.element_size() for h in host_in)
        d2h = sum(h.numel() * h.element_size() for h in slots[0]["h_out"])
        pat_bytes = sum(h.numel() * h.element_size() for h in slots[0]["h_pat"])
        tally = {"steps": 0, "pattern_reads": 0}

        def pieces(pairs):
            """(destination, source) pairs cut into ncs lists of flat slices of about equal bytes."""
            flat = [(a.view(-1), b.view(-1)) for a, b in pairs]
            total = sum(a.numel() * a.element_size() for a, _ in flat)
            out, acc, k = [[] for _ in range(ncs)], 0, 0
            for a, b in flat:
                n, es, i = a.numel(), a.element_size(), 0
                while i < n:
                    room = (k + 1) * total // ncs - acc  # bytes left for list k
                    take = n - i if k == ncs - 1 else max(1, min(n - i, room // es))
                    out[k].append((a[i:i + take], b[i:i + take]))
                    i += take
                    acc += take * es
                    if k < ncs - 1 and acc >= (k + 1) * total // ncs:
                        k += 1
            return out

        for sl in slots:
            sl["in_pieces"] = pieces(list(zip(sl["d_in"], host_in)))
            sl["out_pieces"] = pieces(list(zip(sl["h_out"], sl["outs"])))

        def collect(sl):
            """The slot's last step fully on the host: its copies complete, and its pattern read back
            if that step's rebuild changed it (before the slot's next rebuild overwrites it)."""
            for e in sl["ev"]["out"]:
                e.synchronize()
            if int(sl["h_out"][2][0]) or int(sl["h_out"][2][1]):
                with torch.cuda.stream(s_out[0]):
                    for h, d in zip(sl["h_pat"], sl["pat"]):
                        h.copy_(d, non_blocking=True)
                s_out[0].synchronize()
                tally["pattern_reads"] += 1

        def e2e_step():
            sl = slots[tally["steps"] % nslots]
            tally["steps"] += 1
            ev = sl["ev"]
            if sl["used"]:
                collect(sl)
            for q, st in enumerate(s_in):
                if sl["used"]:
                    st.wait_event(ev["comp"])    # the slot's previous compute has read its inputs
                with torch.cuda.stream(st):
                    for d, h in sl["in_pieces"][q]:
                        d.copy_(h, non_blocking=True)
                    ev["in"][q].record(st)
                stream.wait_event(ev["in"][q])
            if sl["used"]:
                for e in ev["out"]:
                    stream.wait_event(e)         # the slot's previous outputs have been read back
            with torch.cuda.stream(stream):
                compute(sl["sp"], sl["A"], sl["X"], sl["Y"], sl["M"], sl["XY"], sl["CM"])
                ev["comp"].record(stream)
            for q, st in enumerate(s_out):
                st.wait_event(ev["comp"])
                with torch.cuda.stream(st):
                    for h, d in sl["out_pieces"][q]:
                        h.copy_(d, non_blocking=True)
                    ev["out"][q].record(st)
            sl["used"] = True

        for k in range(nslots):
            e2e_step()
        torch.cuda.synchronize()
        # three windows of ksteps steps each; the median window is the figure (the host side of the
        # copies is shared with other work on the machine, and one stall can double a short window)
        ksteps = max(3, min(args.steps, 20))
        windows = []
        timed_steps, timed_reads = 0, tally["pattern_reads"]
        for w in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for st in s_in[1:]:
                st.wait_stream(s_in[0])
            a.record(s_in[0])
            for k in range(ksteps):
                e2e_step()
            for st in s_out[1:]:
                s_out[0].wait_stream(st)
            b.record(s_out[0])
            b.synchronize()
            windows.append(a.elapsed_time(b) / ksteps)
            timed_steps += ksteps
        for sl in slots:  # the steps still in flight are collected (and counted) too
            collect(sl)
        timed_reads = tally["pattern_reads"] - timed_reads
        e2e_ms = sorted(windows)[1]
        if dist:
            e2e_ms = max_over_ranks(e2e_ms, dev)
        e2e = {"value": job_throughput(mesh.ncell, world, e2e_ms), "unit": "cells/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h + pat_bytes * timed_reads / timed_steps, "ms_per_step": e2e_ms,
               "windows_ms_per_step": windows, "window_steps": ksteps,
               "outputs": "every step: CSR values, y and the rebuild's two flags (column tracking on: the row pass "
                          "compares each column it writes in place); rowptr and colidx after a rebuild "
                          f"that reports a change ({timed_reads} of {timed_steps} timed steps; "
                          f"{pat_bytes} bytes each), so the host holds the current pattern after every step",
               "pipelining": f"copies of neighbouring steps overlap the compute (three device slots; each direction's "
                             f"copies cut into {ncs} pieces on {ncs} streams)",
               "host_cpus": host_cpus or "unchanged (no local CPU list in sysfs)"}
        fe.sync(ctx)

    # ------------------------------------------------------------------- stored element matrices
    # The stored-matrix alternative to the matrix-free action, timed after the steps and outside them:
    # fe_elem_matrices once (every cell's upper triangle in FP64, entry-major), then fe_action_stored
    # per application.  Its result is checked against the step's matrix-free action (in Y).
    stored = None
    if not pull and not args.no_stored:
        nd_s = counts_per_cell(wl["dim"], wl["p"])[0]
        nup = nd_s * (nd_s + 1) // 2
        t_ke = torch.empty((nup, mesh.ncell), dtype=torch.float64, device=dev)
        t_y2 = torch.zeros_like(t_x)
        Y2 = fe.dat_create(ctx, nodes, t_y2)
        with torch.cuda.stream(stream):
            for _ in range(2):
                fe.elem_matrices(ctx, K, cells, t_ke, XY, CM)
                fe.action_stored(ctx, K, cells, t_ke, X, Y2, M, zero_first=True)
        fe.sync(ctx)
        reps = 20
        se = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        with torch.cuda.stream(stream):
            se[0].record(stream)
            fe.elem_matrices(ctx, K, cells, t_ke, XY, CM)
            se[1].record(stream)
            for _ in range(reps):
                fe.action_stored(ctx, K, cells, t_ke, X, Y2, M, zero_first=True)
            se[2].record(stream)
        fe.sync(ctx)
        st_ms, sa_ms = se[0].elapsed_time(se[1]), se[1].elapsed_time(se[2]) / reps
        ke_bytes = nup * 8 * mesh.ncell
        sa_bytes = ke_bytes + mesh.ncell * nd_s * 4 + 2 * nn * 8
        ymax = float(t_y.abs().max())
        stored = {"elem_matrices_ms": st_ms, "action_ms": sa_ms, "action_reps": reps, "stored_bytes": ke_bytes,
                  "action_bytes": sa_bytes, "action_gbs": sa_bytes / (sa_ms / 1e3) / 1e9,
                  "max_diff_vs_matrix_free": float((t_y2 - t_y).abs().max()) / (ymax if ymax > 0 else 1.0),
                  "note": "not part of the step: stored matrices trade HBM for the element arithmetic of each action"}
        del t_ke

    # ------------------------------------------------------------------- roofline of the dominant kernel
    peaks, src = _peaks()
    nd, fl_mat, fl_act = counts_per_cell(wl["dim"], wl["p"])
    ncell = mesh.ncell
    bytes_mat = ncell * (nd * 4 + (wl["dim"] + 1) * 4) + mesh.nvert * wl["dim"] * 8 + nnz * 8
    bytes_act = ncell * (nd * 4 + (wl["dim"] + 1) * 4) + mesh.nvert * wl["dim"] * 8 + 2 * nn * 8
    # sparsity build, the method's own bytes: the map read once, rowptr, colidx and the lookup table
    # written once (the incidence lists the design builds on the way are overhead, not counted)
    bytes_sp = ncell * nd * 4 + (nn + 1) * 8 + nnz * 4 + ncell * nd * nd
    if fuse[0]:
        # one pass: the maps and coordinates read once, the zeros, the CSR values, x read, y written;
        # the FP64 work of one element matrix and its nd^2 products with x_e per cell
        bytes_fused = bytes_mat + nnz * 8 + 3 * nn * 8
        kern = {
            "sparsity": {"ms": phase_ms[0], "bytes": bytes_sp},
            "assemble_action": {"ms": phase_ms[2], "bytes": bytes_fused, "flops": ncell * fl_act,
                                "includes": "Mat and y zeros, assembly, matrix-free action (fe_assemble_mat_action)"},
        }
    else:
        kern = {
            "sparsity": {"ms": phase_ms[0], "bytes": bytes_sp},
            "zero": {"ms": phase_ms[1], "bytes": nnz * 8 if not pull else 0},
            "assemble": {"ms": phase_ms[2], "bytes": bytes_mat, "flops": ncell * fl_mat},
            "action": {"ms": phase_ms[3], "bytes": bytes_act, "flops": ncell * fl_act},
        }
    for k, v in kern.items():
        if "bytes" in v and v["ms"] > 0 and v["bytes"] > 0:
            v["gbs"] = v["bytes"] / (v["ms"] / 1e3) / 1e9
            v["hbm_frac"] = v["gbs"] / peaks["hbm_gbs"]
        if "flops" in v and v["ms"] > 0:
            # FMA-equivalent FP64 rate; a fraction of the FP64 peak only when FP64 executes it
            v["fp64_equiv_tflops"] = v["flops"] / (v["ms"] / 1e3) / 1e12
            if args.precision == "fp64":
                v["fp64_frac"] = v["fp64_equiv_tflops"] / FP64_PEAK_TFLOPS
    dom = max(kern, key=lambda k: kern[k]["ms"])
    dk = kern[dom]
    fp64_bound = "flops" in dk and dk["flops"] / (FP64_PEAK_TFLOPS * 1e12) > dk["bytes"] / (peaks["hbm_gbs"] * 1e9)
    if args.precision == "fp64" and fp64_bound:
        roof = {"bound": "alu", "achieved": dk["fp64_equiv_tflops"], "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": dk["fp64_frac"], "kernel": dom, "peak_source": "derived FP64: 152 SMs x 2 FMA/clk x 2.07 GHz"}
    else:
        roof = {"bound": "hbm", "achieved": dk["gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": dk["hbm_frac"], "kernel": dom, "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"}
    # the captured traffic is that of the P2 64^3 workload; other meshes report none
    tr = TRAFFIC.get((dom, args.strategy, args.precision)) or TRAFFIC.get((dom, None, None))
    if args.workload != "p2-3d" or args.n:
        tr = None
    src_file = "fe_sparsity.cu" if dom == "sparsity" else "fe_kernels.cuh"
    fresh = bool(tr) and tr[1] == _src_hash(src_file)
    roof["traffic"] = tr[0] if fresh else None
    roof["binding"] = tr[2] if fresh else None
    # every phase against its own binding roofline, beside the dominant one
    roof["per_kernel"] = {k: ({"bound": "alu", "frac": v["fp64_frac"], "unit": "FP64 TFLOP/s"}
                              if "fp64_frac" in v and v["flops"] / (FP64_PEAK_TFLOPS * 1e12) >
                              v["bytes"] / (peaks["hbm_gbs"] * 1e9) else
                              {"bound": "hbm", "frac": v.get("hbm_frac")}) for k, v in kern.items()}
    out = {
        "metric": METRIC, "value": job_throughput(ncell, world, ms_step), "unit": "cells/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32x2 element / f64 accumulate", "data": "synthetic",
        "config": {"workload": wl["name"], "cells_per_gpu": ncell, "dofs": nn, "nnz": nnz,
                   "strategy": args.strategy,
                   "schedule": (("action on a second stream, concurrent with the Mat zero and assembly" if beside_asm
                                 else "Mat zero and action on a second stream, concurrent with the sparsity rebuild"
                                 if side is not None else
                                 "serial on one stream: sparsity rebuild, then the Mat and y zeros, assembly and "
                                 "matrix-free action in one pass (fe_assemble_mat_action: each cell's element "
                                 "matrix built once for both outputs)" if fuse[0] else
                                 "serial on one stream") +
                                (", one CUDA graph per step (phases from a launch-by-launch pass)"
                                 if graph is not None else "")),
                   "precision": ("element tensors in FP32 pairs (double-float), FP64 global accumulation"
                                 if args.precision == "f32x2" else "FP64 throughout"),
                   "parallelism": f"replicas x{world} (independent meshes, no collective)",
                   "l2": ("inputs larger than L2 (CSR values + lookup table ~650 MB), no flush" if flush is None else
                          "L2 flushed between steps (256 MB written outside the timed intervals)")},
        "roofline": roof, "kernels": kern, "step_ms": step_stats, "gpu_launches": launches, "wall_s_timed": wall,
        "clocks": clk.summary(), "e2e": e2e, "stored_action": stored, "f32x2_step": f32x2,
    }
    if out["clocks"].get("sm_mhz"):
        out["clocks"]["ms_x_mhz"] = ms_step * out["clocks"]["sm_mhz"]
    return out, (mesh, cmap, nn, x)


# ------------------------------------------------------------------------------ batched workload

# ------------------------------------------------------------------------------ wave steps

def run_wave(args, wl, rank, world):
    import torch
    from paper_1501_01809_gb300 import build as fb
    from paper_1501_01809_gb300 import fe
    from paper_1501_01809_gb300 import meshgen as mg
    fb.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    mesh, cmap, nn, _ = make_inputs(wl)
    bc = mg.face_nodes(mesh, 1, 1, 0)
    stream = torch.cuda.Stream(dev)
    ctx = fe.ctx_create(dev.index, stream=stream)
    prec = {"fp64": fe.PREC_FP64, "f32x2": fe.PREC_F32X2}[args.precision]
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in
         dict(map=cmap, cv=mesh.cell_vertex, xy=mesh.coords, bc=bc, one=np.ones(nn)).items()}
    phi = torch.zeros(nn, dtype=torch.float64, device=dev)
    pv = torch.zeros(nn, dtype=torch.float64, device=dev)
    mass = torch.zeros(nn, dtype=torch.float64, device=dev)
    dt = wl["dt"]
    with torch.cuda.stream(stream):
        cells, nodes, verts = fe.set_create(ctx, mesh.ncell), fe.set_create(ctx, nn), fe.set_create(ctx, mesh.nvert)
        M, CM = fe.map_create(ctx, cells, nodes, t["map"]), fe.map_create(ctx, cells, verts, t["cv"])
        XY = fe.dat_create(ctx, verts, t["xy"])
        PHI, P = fe.dat_create(ctx, nodes, phi), fe.dat_create(ctx, nodes, pv)
        ONE, MASS = fe.dat_create(ctx, nodes, t["one"]), fe.dat_create(ctx, nodes, mass)
        sp = fe.sparsity_build(ctx, M, M)
        ks = fe.kernel_create(ctx, fe.FORM_SOURCE, wl["dim"], 1, coeff_degree=1, strategy=fe.STRATEGY_PULL)
        fe.assemble_vec(ctx, ks, cells, MASS, M, XY, CM, [(ONE, M)], zero_first=True, sp=sp)
        kl = fe.kernel_create(ctx, fe.FORM_LAPLACE, wl["dim"], 1, precision=prec)
    fe.wave_steps(ctx, kl, cells, PHI, P, mass, t["bc"], M, XY, CM, sp, 0.0, dt, args.warmup)
    fe.sync(ctx)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        a.record(stream)
        fe.wave_steps(ctx, kl, cells, PHI, P, mass, t["bc"], M, XY, CM, sp, args.warmup * dt, dt, args.steps)
        b.record(stream)
        b.synchronize()
    ms = a.elapsed_time(b) / args.steps
    if world > 1:
        ms = max_over_ranks(ms, dev)
    fe.sync(ctx)
    # e2e: every time step takes (phi, p) from pinned host memory and returns them
    h_in = [torch.empty(nn, dtype=torch.float64, pin_memory=True).copy_(x.cpu()) for x in (phi, pv)]
    h_out = [torch.empty(nn, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    ke = max(3, min(args.steps, 50))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(ke):
        with torch.cuda.stream(stream):
            phi.copy_(h_in[0], non_blocking=True)
            pv.copy_(h_in[1], non_blocking=True)
            fe.wave_steps(ctx, kl, cells, PHI, P, mass, t["bc"], M, XY, CM, sp, 0.0, dt, 1)
            h_out[0].copy_(phi, non_blocking=True)
            h_out[1].copy_(pv, non_blocking=True)
    e1.record(stream)
    e1.synchronize()
    e2e_ms = e0.elapsed_time(e1) / ke
    peaks, src = _peaks()
    # algorithmic bytes per time step: maps (4 + 4 ints per cell), coordinates and phi gathered once,
    # p, phi read and written, mass and the boundary flags read once
    byt = mesh.ncell * 32 + mesh.nvert * 24 + nn * (8 + 16 + 16 + 8 + 1)
    gbs = byt / (ms / 1e3) / 1e9
    out = {"metric": "cells/s stepped (explicit wave: action + lumped-mass updates per time step)",
           "value": job_throughput(mesh.ncell, world, ms), "unit": "cells/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32x2 element / f64 accumulate", "data": "synthetic",
           "config": {"workload": wl["name"], "cells_per_gpu": mesh.ncell, "nodes": nn,
                      "precision": ("action element tensors in FP32 pairs, FP64 state" if args.precision == "f32x2"
                                    else "FP64 throughout"),
                      "step": "one time step", "parallelism": f"replicas x{world}",
                      "l2": "state and maps larger than L2 in total; no flush"},
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                        "kernel": "time step (k_action_elem<3,1,LAPLACE> + k_wave_row)",
                        "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"},
           "gpu_launches": 2 * args.steps + 1, "clocks": clk.summary(),
           "e2e": {"value": job_throughput(mesh.ncell, world, e2e_ms), "unit": "cells/s",
                   "h2d_bytes_per_step": 16 * nn, "d2h_bytes_per_step": 16 * nn, "ms_per_step": e2e_ms}}
    return out, (mesh, cmap, nn, bc)


def wave_cpu_sample(wl, inputs, budget_s):
    """Oracle wave steps on the workload mesh, one step at a time, until budget_s seconds."""
    import oracle as O
    mesh, cmap, nn, bc = inputs
    # one call (its lumped mass once, then the steps); the step count from a one-step probe
    t0 = time.perf_counter()
    O.wave_steps(wl["dim"], 1, cmap, mesh.coords, mesh.cell_vertex, nn, np.zeros(nn), np.zeros(nn), 0.0, wl["dt"], 1,
                 is_bc=bc)
    probe = time.perf_counter() - t0
    steps = max(1, int(budget_s / max(probe, 1e-3)))
    t0 = time.perf_counter()
    O.wave_steps(wl["dim"], 1, cmap, mesh.coords, mesh.cell_vertex, nn, np.zeros(nn), np.zeros(nn), 0.0, wl["dt"],
                 steps, is_bc=bc)
    return steps * mesh.ncell, time.perf_counter() - t0


# ------------------------------------------------------------------------------ P1 roofline sweep

def run_p1_sweep(args, wl, rank, world):
    """Assembly (zero + Mat) and action of P1 Helmholtz on n x n squares for several n: the P1 roofline
    behaviour as the mesh outgrows L2.  Sparsity built once per n (outside the timed loop)."""
    import torch
    from paper_1501_01809_gb300 import build as fb
    from paper_1501_01809_gb300 import fe
    fb.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    ctx = fe.ctx_create(dev.index, stream=stream)
    prec = {"fp64": fe.PREC_FP64, "f32x2": fe.PREC_F32X2}[args.precision]
    peaks, src = _peaks()
    rows = []
    clk = ClockSampler(dev.index)
    clk.__enter__()
    for n in wl["ns"]:
        w = dict(wl, n=n)
        mesh, cmap, nn, x = make_inputs(w)
        t = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in
             dict(map=cmap, cv=mesh.cell_vertex, xy=mesh.coords, x=x).items()}
        ty = torch.zeros_like(t["x"])
        with torch.cuda.stream(stream):
            cells, nodes, verts = fe.set_create(ctx, mesh.ncell), fe.set_create(ctx, nn), fe.set_create(ctx, mesh.nvert)
            M, CM = fe.map_create(ctx, cells, nodes, t["map"]), fe.map_create(ctx, cells, verts, t["cv"])
            XY, X, Y = fe.dat_create(ctx, verts, t["xy"]), fe.dat_create(ctx, nodes, t["x"]), fe.dat_create(ctx, nodes, ty)
            K = fe.kernel_create(ctx, fe.FORM_HELMHOLTZ, 2, 1, precision=prec, strategy=fe.STRATEGY_PUSH)
            sp = fe.sparsity_build(ctx, M, M)
            A = fe.mat_create(ctx, sp)
        nnz = fe.sparsity_csr(sp)[2]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        for _ in range(args.warmup):
            fe.assemble_mat(ctx, K, cells, A, XY, CM, zero_first=True)
            fe.action(ctx, K, cells, X, Y, M, XY, CM, zero_first=True)
        fe.sync(ctx)
        reps = max(3, min(args.steps, 50))
        ev[0].record(stream)
        for _ in range(reps):
            fe.assemble_mat(ctx, K, cells, A, XY, CM, zero_first=True)
        ev[1].record(stream)
        for _ in range(reps):
            fe.action(ctx, K, cells, X, Y, M, XY, CM, zero_first=True)
        ev[2].record(stream)
        ev[2].synchronize()
        ms_a, ms_x = ev[0].elapsed_time(ev[1]) / reps, ev[1].elapsed_time(ev[2]) / reps
        # algorithmic bytes: map 12 + coordinate map 12 per cell, coordinates once, CSR values written
        # once (zero + INC counted once), x read and y written once for the action
        b_a = mesh.ncell * 24 + mesh.nvert * 16 + nnz * 8
        b_x = mesh.ncell * 24 + mesh.nvert * 16 + 2 * nn * 8
        rows.append({"n": n, "cells": mesh.ncell, "nnz": nnz, "assemble_ms": ms_a, "action_ms": ms_x,
                     "assemble_cells_per_s": mesh.ncell / (ms_a / 1e3), "action_cells_per_s": mesh.ncell / (ms_x / 1e3),
                     "assemble_hbm_frac": b_a / (ms_a / 1e3) / 1e9 / peaks["hbm_gbs"],
                     "action_hbm_frac": b_x / (ms_x / 1e3) / 1e9 / peaks["hbm_gbs"]})
        del A, sp
    clk.__exit__(None, None, None)
    big = rows[-1]
    gbs = (big["cells"] * 24 + (big["n"] + 1) ** 2 * 16 + big["nnz"] * 8) / (big["assemble_ms"] / 1e3) / 1e9
    out = {"metric": "cells/s assembled (P1 CSR assembly incl. zero), labelled extra sweep", "value":
           world * big["assemble_cells_per_s"], "unit": "cells/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": big["assemble_ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32x2 element / f64 accumulate", "data": "synthetic",
           "config": {"workload": wl["name"], "sweep": rows, "precision": args.precision,
                      "parallelism": f"replicas x{world}", "l2": "largest n: inputs larger than L2"},
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                        "kernel": f"k_zero_f64 + k_mat_push<2,1,HELMHOLTZ> at n={big['n']}",
                        "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"},
           "gpu_launches": 2 * max(3, min(args.steps, 50)), "clocks": clk.summary(), "e2e": None}
    return out


# ------------------------------------------------------------------------------ P4 kappa precision study

def run_p4(args, wl, rank, world):
    """Zero + assembly of the P4 kappa-diffusion Mat (sparsity built once) for the element-tensor
    precisions; the step is the tensor-core variant; errors against the FP64 variant."""
    import torch
    from paper_1501_01809_gb300 import build as fb
    from paper_1501_01809_gb300 import fe
    from paper_1501_01809_gb300 import meshgen as mg
    fb.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    mesh, cmap, nn, _ = make_inputs(wl)
    kap = mg.lognormal_dat(mesh.nvert, wl["kappa_seed"])
    stream = torch.cuda.Stream(dev)
    ctx = fe.ctx_create(dev.index, stream=stream)
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in
         dict(map=cmap, cv=mesh.cell_vertex, xy=mesh.coords, kap=kap).items()}
    with torch.cuda.stream(stream):
        cells, nodes, verts = fe.set_create(ctx, mesh.ncell), fe.set_create(ctx, nn), fe.set_create(ctx, mesh.nvert)
        M, CM = fe.map_create(ctx, cells, nodes, t["map"]), fe.map_create(ctx, cells, verts, t["cv"])
        XY, KAP = fe.dat_create(ctx, verts, t["xy"]), fe.dat_create(ctx, verts, t["kap"])
        sp = fe.sparsity_build(ctx, M, M)
        A = fe.mat_create(ctx, sp)
    nnz = fe.sparsity_csr(sp)[2]
    vals = fe.mat_values(A)
    res, outs = {}, {}
    variants = [("tf32x3", fe.PREC_TF32X3), ("fp32", fe.PREC_FP32), ("fp64", fe.PREC_FP64)]
    clk_summary = None
    for name, prec in variants:
        K = fe.kernel_create(ctx, fe.FORM_KAPPA_DIFFUSION, 2, 4, precision=prec)
        for _ in range(args.warmup):
            fe.assemble_mat(ctx, K, cells, A, XY, CM, [(KAP, CM)], zero_first=True)
        fe.sync(ctx)
        steps = args.steps if name == "tf32x3" else max(3, min(args.steps, 20))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev.index) as clk:
            a.record(stream)
            for _ in range(steps):
                fe.assemble_mat(ctx, K, cells, A, XY, CM, [(KAP, CM)], zero_first=True)
            b.record(stream)
            b.synchronize()
        if name == "tf32x3":
            clk_summary = clk.summary()
        fe.sync(ctx)
        res[name] = a.elapsed_time(b) / steps
        with torch.cuda.stream(stream):  # copied before the next variant overwrites the values
            outs[name] = vals.clone()
        stream.synchronize()
    ref = outs["fp64"]
    err = {k: float((outs[k] - ref).norm() / ref.norm()) for k in ("tf32x3", "fp32")}
    ms = res["tf32x3"]
    if world > 1:
        ms = max_over_ranks(ms, dev)
    peaks, src = _peaks()
    # algorithmic bytes: map 60 + coordinate map 12 per cell, coordinates and kappa once, CSR values
    # written once (zero + INC counted once)
    byt = mesh.ncell * 72 + mesh.nvert * 24 + nnz * 8
    gbs = byt / (ms / 1e3) / 1e9
    tflop = mesh.ncell * 2 * 18 * 120 * 3 / (ms / 1e3) / 1e12  # three TF32 products per cell
    return {"metric": "cells/s assembled (P4 kappa-diffusion CSR, element tensors on the tensor cores)",
            "value": job_throughput(mesh.ncell, world, ms), "unit": "cells/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "tf32x3", "data": "synthetic",
            "config": {"workload": wl["name"], "cells_per_gpu": mesh.ncell, "dofs": nn, "nnz": nnz,
                       "ms_per_assembly": res, "rel_frobenius_vs_fp64": err,
                       "tensor_tflops_issued": tflop, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (CSR values 789 MB), no flush"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                         "kernel": "k_zero_f64 + k_mat_push_tc_kappa_p4 (the scatter of 225 FP64 values per cell binds; "
                                   "the tensor-core product is a few microseconds)",
                         "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"},
            "gpu_launches": 2 * args.steps, "clocks": clk_summary, "e2e": None}


def make_batch_inputs(wl):
    """Per mesh (n, p, mesh, cell-node map, nodes, f); meshes of equal (n, p) share host arrays only."""
    from paper_1501_01809_gb300 import meshgen as mg
    ns, ps = mg.batch_mesh_sizes(wl["count"], wl["seed"], wl["lo"], wl["hi"])
    cache, out = {}, []
    for i, (n, p) in enumerate(zip(ns, ps)):
        key = (int(n), int(p))
        if key not in cache:
            mesh = mg.unit_square_mesh(key[0])
            cmap, nn = mg.cell_node_map(mesh, key[1])
            cache[key] = (mesh, cmap, nn)
        mesh, cmap, nn = cache[key]
        out.append((key[0], key[1], mesh, cmap, nn, mg.uniform_dat(nn, 1000 + i)))
    return out


def _concat_to_device(arrays, dev):
    """One device buffer holding all arrays back to back; returns (buffer, [views])."""
    import torch
    flat = np.concatenate([a.ravel() for a in arrays])
    buf = torch.from_numpy(flat).to(dev)
    views, off = [], 0
    for a in arrays:
        views.append(buf[off:off + a.size].view(a.shape))
        off += a.size
    return buf, views


def run_batch(args, wl, rank, world):
    import torch
    from paper_1501_01809_gb300 import build as fb
    from paper_1501_01809_gb300 import fe

    fb.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    meshes = make_batch_inputs(wl)
    stream = torch.cuda.Stream(dev)
    ctx = fe.ctx_create(dev.index, stream=stream)
    prec = {"fp64": fe.PREC_FP64, "f32x2": fe.PREC_F32X2}[args.precision]
    kmat = {p: fe.kernel_create(ctx, fe.FORM_HELMHOLTZ, 2, p, precision=prec) for p in (1, 2)}
    kvec = {p: fe.kernel_create(ctx, fe.FORM_SOURCE, 2, p, coeff_degree=p, precision=prec) for p in (1, 2)}
    host = {"map": [m[3] for m in meshes], "cv": [m[2].cell_vertex for m in meshes],
            "xy": [m[2].coords for m in meshes], "f": [m[5] for m in meshes]}
    bufs, views = {}, {}
    for k, arrs in host.items():
        bufs[k], views[k] = _concat_to_device(arrs, dev)
    items, objs = [], []
    ncell_tot = nnz_tot = bytes_alg = 0
    with torch.cuda.stream(stream):
        for i, (n, p, mesh, cmap, nn, f) in enumerate(meshes):
            cells, nodes, verts = fe.set_create(ctx, mesh.ncell), fe.set_create(ctx, nn), fe.set_create(ctx, mesh.nvert)
            M = fe.map_create(ctx, cells, nodes, views["map"][i])
            CM = fe.map_create(ctx, cells, verts, views["cv"][i])
            XY = fe.dat_create(ctx, verts, views["xy"][i])
            F = fe.dat_create(ctx, nodes, views["f"][i])
            sp = fe.sparsity_build(ctx, M, M)
            nnz = fe.sparsity_csr(sp)[2]
            items.append(dict(kmat=kmat[p], kvec=kvec[p], cells=cells, sp=sp, coords=XY, coord_map=CM, f=(F, M)))
            objs.append((cells, nodes, M, CM, XY, F, sp, p))
            nd = 3 if p == 1 else 6
            ncell_tot += mesh.ncell
            nnz_tot += nnz
            # algorithmic bytes: maps and coordinates read once, f read once, CSR values and RHS written once
            bytes_alg += mesh.ncell * (nd + 3) * 4 + mesh.nvert * 16 + nn * 8 + nnz * 8 + nn * 8
        B = fe.batch_create(ctx, items)
    fe.sync(ctx)
    tile, grid, tune_ms = fe.batch_tune(B, reps=3)

    def time_loop(fn, k):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / k

    step = lambda: fe.batch_assemble(B, use_graph=True)
    for _ in range(args.warmup):
        step()
    fe.sync(ctx)
    dist = world > 1
    if dist:
        import torch.distributed as td
        td.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        t0 = time.perf_counter()
        ms_step = time_loop(step, args.steps)
        wall = time.perf_counter() - t0
    if dist:
        td.barrier()
        ms_step = max_over_ranks(ms_step, dev)
    fe.sync(ctx)
    # the same batch without the graph, and the plain path: one Mat zero + one Mat launch + one RHS
    # launch per mesh (its own Mat and RHS), both on the same stream
    ksmall = max(3, min(args.steps, 20))
    eager_ms = time_loop(lambda: fe.batch_assemble(B, use_graph=False), ksmall)
    mats, rhs = [], []
    for (cells, nodes, M, CM, XY, F, sp, p) in objs:
        mats.append(fe.mat_create(ctx, sp))
        t_b = torch.empty(fe.sparsity_csr(sp)[0], dtype=torch.float64, device=dev)
        rhs.append((t_b, fe.dat_create(ctx, nodes, t_b)))

    def plain():
        for (cells, nodes, M, CM, XY, F, sp, p), A, (_, Bv) in zip(objs, mats, rhs):
            fe.mat_zero(A)
            fe.assemble_mat(ctx, kmat[p], cells, A, XY, CM)
            fe.assemble_vec(ctx, kvec[p], cells, Bv, M, XY, CM, [(F, M)], zero_first=True)

    plain()
    fe.sync(ctx)
    plain_ms = time_loop(plain, ksmall)
    fe.sync(ctx)
    # batched results equal the plain ones (spot check of the largest mesh's RHS, relative 1e-12)
    big = int(np.argmax([m[2].ncell for m in meshes]))
    rb = fe.batch_values(B, big)[1]
    drift = float((rb - rhs[big][0]).abs().max() / max(1e-300, float(rhs[big][0].abs().max())))

    e2e = None
    if not args.no_e2e:
        vals_all, rhs_all = fe.batch_buffers(B)
        h_in = [(torch.empty(t.shape, dtype=t.dtype, pin_memory=True).copy_(t.cpu()), t) for t in bufs.values()]
        h_out = [(torch.empty(t.shape, dtype=t.dtype, pin_memory=True), t) for t in (vals_all, rhs_all)]
        h2d = sum(h.numel() * h.element_size() for h, _ in h_in)
        d2h = sum(h.numel() * h.element_size() for h, _ in h_out)

        def e2e_step():
            with torch.cuda.stream(stream):
                for h, d in h_in:
                    d.copy_(h, non_blocking=True)
                step()
                for h, d in h_out:
                    h.copy_(d, non_blocking=True)

        e2e_step()
        stream.synchronize()
        e2e_ms = time_loop(e2e_step, ksmall)
        e2e = {"value": world * ncell_tot / (e2e_ms / 1e3), "unit": "cells/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms}
        fe.sync(ctx)

    peaks, src = _peaks()
    gbs = bytes_alg / (ms_step / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
            "kernel": "batch step (k_batch_zero + k_batch_assemble, one graph)", "traffic": None,
            "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"}
    out = {
        "metric": METRIC_BATCH, "value": job_throughput(ncell_tot, world, ms_step), "unit": "cells/s",
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32x2 element / f64 accumulate", "data": "synthetic",
        "config": {"workload": wl["name"], "meshes": len(meshes), "cells_per_gpu": ncell_tot, "nnz": nnz_tot,
                   "precision": ("element tensors in FP32 pairs (double-float), FP64 global accumulation"
                                 if args.precision == "f32x2" else "FP64 throughout"),
                   "tuned": {"tile_cells": tile, "grid": grid, "ms": tune_ms},
                   "batched_eager_ms": eager_ms, "plain_per_mesh_ms": plain_ms,
                   "plain_cells_per_s": ncell_tot / (plain_ms / 1e3), "speedup_vs_plain": plain_ms / ms_step,
                   "plain_launches_per_step": 3 * len(meshes), "max_rel_diff_vs_plain_rhs": drift,
                   "parallelism": f"replicas x{world} (independent batches, no collective)",
                   "l2": f"inputs larger than L2 (CSR values {8 * nnz_tot / 1e9:.2f} GB), no flush"},
        "roofline": roof, "gpu_launches": 2 * args.steps, "wall_s_timed": wall, "clocks": clk.summary(), "e2e": e2e,
    }
    return out, meshes


# ------------------------------------------------------------------------------ serving workload

def make_serve_inputs(wl):
    """Per request (n, p, k, m, cell-node map, mesh, nodes, f, boundary mask); meshes cached by (n, p)."""
    from paper_1501_01809_gb300 import meshgen as mg
    reqs = mg.serve_requests(wl["count"], wl["seed"], 1.0, wl["lo"], wl["hi"])
    cache, out = {}, []
    for (t, n, p, k, m) in reqs:
        if (n, p) not in cache:
            mesh = mg.unit_square_mesh(n)
            cmap, nn = mg.cell_node_map(mesh, p)
            cache[(n, p)] = (mesh, cmap, nn, mg.boundary_nodes(mesh, p))
        mesh, cmap, nn, bc = cache[(n, p)]
        f, _ = mg.manufactured_sine(mesh, p, k, m)
        out.append(dict(t1=t, n=n, p=p, k=k, m=m, mesh=mesh, cmap=cmap, nn=nn, f=f, bc=bc))
    return out


def _serve_once(fe, ctx, wl, reqs, rate, max_active, keyed=None):
    """One run of the request loop; arrival times are the unit-rate draws divided by rate (0: all at once).
    keyed (default: the served configuration, max_active > 1): requests name their mesh by (n, p), so
    that requests on the same mesh share its device copy and sparsity; the plain path builds each
    request's mesh for that request alone."""
    keyed = max_active > 1 if keyed is None else keyed
    srv = fe.server_create(ctx, wl["budget"], max_active=max_active, iters_per_tick=wl["tick"], rtol=1e-8)
    ids, xs = [], []
    for r in reqs:
        x = np.empty(r["nn"])
        t = r["t1"] / rate if rate > 0 else 0.0
        key = (r["n"] << 4 | r["p"]) if keyed else 0
        ids.append(fe.server_submit(srv, r["p"], r["cmap"], r["mesh"].cell_vertex, r["mesh"].coords, r["f"], r["bc"],
                                    x, t, mesh_key=key))
        xs.append(x)
    fe.server_run(srv)
    res = [fe.server_result(srv, i) for i in ids]
    st = fe.server_stats(srv)
    srv.destroy()
    arr = np.array([r["t1"] / rate if rate > 0 else 0.0 for r in reqs])
    lat = np.array([q["finished_s"] for q in res]) - arr
    ok = all(q["status"] == fe.SOLVE_CONVERGED for q in res)
    return {"rate_req_s": rate, "solves_per_s": len(reqs) / st["run_s"], "run_s": st["run_s"],
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_iters": float(np.mean([q["iters"] for q in res])), "all_converged": ok,
            "peak_bytes": st["peak_bytes"], "cg_launches": st["cg_launches"],
            "mesh_cache": {"hits": st["cache_hits"], "misses": st["cache_misses"], "evictions": st["cache_evictions"],
                           "sparsity_builds": st["sparsity_builds"]},
            "host_s": {"admit": st["admit_s"], "tick": st["tick_s"], "retire": st["retire_s"]}}, xs


def run_serve(args, wl, rank, world):
    import torch
    from paper_1501_01809_gb300 import build as fb
    from paper_1501_01809_gb300 import fe
    from paper_1501_01809_gb300 import meshgen as mg

    fb.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    reqs = make_serve_inputs(wl)
    stream = torch.cuda.Stream(dev)
    ctx = fe.ctx_create(dev.index, stream=stream)
    # warm-up: a few small requests through both paths
    small = [r for r in reqs if r["n"] <= 40][:4] or reqs[:2]
    for _ in range(args.warmup):
        _serve_once(fe, ctx, wl, small, 0.0, wl["max_active"])
        _serve_once(fe, ctx, wl, small, 0.0, 1)
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sat, x_mix = _serve_once(fe, ctx, wl, reqs, 0.0, wl["max_active"])
        b.record(stream)
        b.synchronize()
        dev_ms = a.elapsed_time(b)
        plain_sat, x_one = _serve_once(fe, ctx, wl, reqs, 0.0, 1)
        identical = all(np.array_equal(u, v) for u, v in zip(x_mix, x_one))
        sweep = []
        for frac in (0.25, 0.5, 0.75, 0.9):
            rate = frac * sat["solves_per_s"]
            served, _ = _serve_once(fe, ctx, wl, reqs, rate, wl["max_active"])
            plain, _ = _serve_once(fe, ctx, wl, reqs, rate, 1)
            sweep.append({"rate_req_s": rate, "served": served, "plain": plain})
    # CG iteration of the largest system alone: the dominant kernels, timed with CUDA events
    big = max(reqs, key=lambda r: r["nn"] * (r["p"] ** 2))
    it_ms, nnz, it_bytes = cg_single_system(fe, ctx, stream, dev, big, 200)
    nn = big["nn"]
    peaks, src = _peaks()
    gbs = it_bytes / (it_ms / 1e3) / 1e9
    h2d = sum(r["cmap"].nbytes + r["mesh"].cell_vertex.nbytes + r["mesh"].coords.nbytes + r["f"].nbytes + r["bc"].nbytes
              for r in reqs)
    d2h = sum(r["nn"] * 8 for r in reqs)
    run_max = max_over_ranks(sat["run_s"], dev) if world > 1 else sat["run_s"]
    out = {
        "metric": METRIC_SERVE, "value": job_throughput(len(reqs), world, 1e3 * run_max), "unit": "solves/s",
        "n_gpus": world,
        "steps": 1, "warmup": args.warmup, "ms_per_step": 1e3 * sat["run_s"] / len(reqs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "requests": len(reqs), "hbm_budget_bytes": wl["budget"],
                   "max_active": wl["max_active"], "iters_per_tick": wl["tick"],
                   "step": "one solve (ms_per_step = run time / requests at saturation)",
                   "gpu_launches_counted": "CG engine launches of the saturated served run (set-up, iterations, "
                                           "polls); each admission adds its sparsity, assembly and elimination "
                                           "launches",
                   "saturation": {"served": sat, "plain_one_at_a_time": plain_sat,
                                  "speedup": sat["solves_per_s"] / plain_sat["solves_per_s"],
                                  "device_ms_served_run": dev_ms},
                   "mixed_equals_alone_bitwise": identical, "rate_sweep": sweep,
                   "parallelism": f"replicas x{world} (independent servers, no collective)",
                   "l2": "each request's data is written and read within its own solve; no flush"},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                     "kernel": f"CG iteration (k_cg_direction_spmv + k_cg_update), largest request alone "
                               f"(P{big['p']} n={big['n']}, {nn} rows, {nnz} nonzeros): {it_ms * 1e3:.1f} us/iteration",
                     "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"},
        "gpu_launches": sat["cg_launches"], "clocks": clk.summary(),
        "e2e": {"value": job_throughput(len(reqs), world, 1e3 * run_max), "unit": "solves/s",
                "h2d_bytes_per_step": h2d // len(reqs),
                "d2h_bytes_per_step": d2h // len(reqs),
                "note": "the served figure is already host to host: meshes copied in, solutions copied out"},
    }
    return out, reqs


SERVE_CPU_MAX_N = 128


def cg_single_system(fe, ctx, stream, dev, req, iters, warm=10):
    """Assemble (pull), eliminate and iterate CG on one request's system alone; returns the mean
    time of one iteration (ms), nnz and the algorithmic bytes of one iteration."""
    import torch
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in
         dict(map=req["cmap"], cv=req["mesh"].cell_vertex, xy=req["mesh"].coords, f=req["f"], bc=req["bc"]).items()}
    nn = req["nn"]
    tb, tx = torch.zeros(nn, dtype=torch.float64, device=dev), torch.zeros(nn, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        cells, nodes, verts = (fe.set_create(ctx, req["mesh"].ncell), fe.set_create(ctx, nn),
                               fe.set_create(ctx, req["mesh"].nvert))
        M, CM = fe.map_create(ctx, cells, nodes, t["map"]), fe.map_create(ctx, cells, verts, t["cv"])
        XY, F = fe.dat_create(ctx, verts, t["xy"]), fe.dat_create(ctx, nodes, t["f"])
        B, X = fe.dat_create(ctx, nodes, tb), fe.dat_create(ctx, nodes, tx)
        sp = fe.sparsity_build(ctx, M, M)
        A = fe.mat_create(ctx, sp)
        kl = fe.kernel_create(ctx, fe.FORM_LAPLACE, 2, req["p"], strategy=fe.STRATEGY_PULL)
        ks = fe.kernel_create(ctx, fe.FORM_SOURCE, 2, req["p"], coeff_degree=req["p"], strategy=fe.STRATEGY_PULL)
        fe.assemble_mat(ctx, kl, cells, A, XY, CM, zero_first=True)
        fe.assemble_vec(ctx, ks, cells, B, M, XY, CM, [(F, M)], zero_first=True, sp=sp)
        fe.dirichlet_apply(ctx, A, B, t["bc"])
        cg = fe.cg_create(ctx, 1)
        fe.cg_add(cg, A, B, X, rtol=1e-30, maxit=1 << 30)
        fe.cg_iterate(cg, warm)
        fe.sync(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fe.cg_iterate(cg, iters)
        e1.record(stream)
        e1.synchronize()
    nnz = fe.sparsity_csr(sp)[2]
    # algorithmic bytes of one iteration (launch A + launch B): values and columns once, slice
    # offsets, z gathered once, p and q read and written (A); p, q, x, r, diag^-1 read, x, r, z
    # written (B)
    it_bytes = nnz * 12 + (nn // 32 + 1) * 8 + nn * 8 + 4 * nn * 8 + 8 * nn * 8
    return e0.elapsed_time(e1) / iters, nnz, it_bytes


def run_cg(args, wl, rank, world):
    """One CG system alone (the largest request of the serving workload): iterations per second."""
    import torch
    from paper_1501_01809_gb300 import build as fb
    from paper_1501_01809_gb300 import fe
    fb.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    reqs = make_serve_inputs(dict(WORKLOADS["serve"]))
    big = max(reqs, key=lambda r: r["nn"] * (r["p"] ** 2))
    stream = torch.cuda.Stream(dev)
    ctx = fe.ctx_create(dev.index, stream=stream)
    with ClockSampler(dev.index) as clk:
        it_ms, nnz, it_bytes = cg_single_system(fe, ctx, stream, dev, big, args.steps, warm=args.warmup)
    if world > 1:
        it_ms = max_over_ranks(it_ms, dev)
    peaks, src = _peaks()
    gbs = it_bytes / (it_ms / 1e3) / 1e9
    return {"metric": "CG iterations/s (one system alone)", "value": world * 1e3 / it_ms, "unit": "iterations/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": it_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"Jacobi-CG iteration on the largest serving request (P{big['p']} n={big['n']}, "
                                   f"{big['nn']} rows, {nnz} nonzeros), SELL-32 SpMV", "step": "one CG iteration",
                       "parallelism": f"replicas x{world}", "l2": "matrix larger than L2"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                         "kernel": "k_cg_direction_spmv + k_cg_update",
                         "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"},
            "gpu_launches": 2 * args.steps, "clocks": clk.summary(), "e2e": None}


def serve_cpu_sample(reqs, budget_s):
    """Oracle on the requests with n <= SERVE_CPU_MAX_N, in arrival order (sparsity, assembly,
    elimination, CG), until budget_s seconds (a single larger solve would take minutes on one core)."""
    import oracle as O
    done, t0 = 0, time.perf_counter()
    small = [q for q in reqs if q["n"] <= SERVE_CPU_MAX_N]
    for r in (small[k % len(small)] for k in range(1 << 30)):
        rp, ci = O.sparsity(r["cmap"], r["cmap"], r["nn"], r["nn"])
        v, _ = O.assemble_mat(2, r["p"], O.LAPLACE, r["cmap"], r["mesh"].coords, r["mesh"].cell_vertex, rp, ci)
        b, _ = O.assemble_vec(2, r["p"], r["p"], r["cmap"], r["nn"], r["mesh"].coords, r["mesh"].cell_vertex, r["f"],
                              r["cmap"])
        v, b = O.dirichlet_apply(rp, ci, v, b, r["bc"])
        O.cg_jacobi(rp, ci, v, b, rtol=1e-8)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return done, time.perf_counter() - t0


def batch_cpu_sample(meshes, budget_s):
    """Oracle on the first meshes of the batch (sparsity + CSR + RHS) until budget_s seconds are spent."""
    import oracle as O
    cells, t0 = 0, time.perf_counter()
    for (n, p, mesh, cmap, nn, f) in meshes:
        rp, ci = O.sparsity(cmap, cmap, nn, nn)
        O.assemble_mat(2, p, O.HELMHOLTZ, cmap, mesh.coords, mesh.cell_vertex, rp, ci)
        O.assemble_vec(2, p, p, cmap, nn, mesh.coords, mesh.cell_vertex, f, cmap)
        cells += mesh.ncell
        if time.perf_counter() - t0 > budget_s:
            break
    return cells, time.perf_counter() - t0


def _oracle_sample(wl, inputs, ncell_sample):
    """Oracle on the first ncell_sample cells of the workload: sparsity + assembly + action."""
    import oracle as O
    mesh, cmap, nn, x = inputs
    c = np.ascontiguousarray(cmap[:ncell_sample])
    cv = np.ascontiguousarray(mesh.cell_vertex[:ncell_sample])
    t0 = time.perf_counter()
    rp, ci = O.sparsity(c, c, nn, nn)
    O.assemble_mat(wl["dim"], wl["p"], O.HELMHOLTZ, c, mesh.coords, cv, rp, ci)
    O.action(wl["dim"], wl["p"], O.HELMHOLTZ, c, mesh.coords, cv, x)
    return time.perf_counter() - t0


def cpu_baseline(wl, inputs, ncell_sample):
    import oracle
    oracle.build()
    _oracle_sample(wl, inputs, min(1024, ncell_sample))  # warm
    dt = _oracle_sample(wl, inputs, ncell_sample)
    return {"value": ncell_sample / dt, "unit": "cells/s", "cores": 1, "kind": "oracle",
            "sample": f"first {ncell_sample} cells of the workload mesh (sparsity + assembly + action), "
                      f"{dt:.1f} s on 1 host core"}


def _oracle_block_worker(task):
    """One process of the all-cores oracle sample: sparsity + assembly + action on its own block of
    cells, inputs memory-mapped from the files the parent wrote.  Returns its seconds of work."""
    d, lo, hi = task
    import oracle as O
    with open(os.path.join(d, "meta.json")) as fh:
        meta = json.load(fh)
    c = np.ascontiguousarray(np.load(os.path.join(d, "cmap.npy"), mmap_mode="r")[lo:hi])
    cv = np.ascontiguousarray(np.load(os.path.join(d, "cv.npy"), mmap_mode="r")[lo:hi])
    coords = np.load(os.path.join(d, "coords.npy"))
    x = np.load(os.path.join(d, "x.npy"))
    t0 = time.perf_counter()
    rp, ci = O.sparsity(c, c, meta["nn"], meta["nn"])
    O.assemble_mat(meta["dim"], meta["p"], O.HELMHOLTZ, c, coords, cv, rp, ci)
    O.action(meta["dim"], meta["p"], O.HELMHOLTZ, c, coords, cv, x)
    return time.perf_counter() - t0


def cpu_baseline_all_cores(wl, inputs, ncell_per_proc, timeout_s=90.0):
    """The oracle sample on every host core this process may use: one spawned process per core, each
    on its own block of ncell_per_proc cells (the blocks' matrices are not merged).  Value = cells of
    all blocks / wall time of the parallel pass."""
    import multiprocessing as mp
    import shutil
    import tempfile
    import oracle
    oracle.build()
    mesh, cmap, nn, x = inputs
    ncpu = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    k = max(1, min(ncpu, mesh.ncell // max(1, ncell_per_proc)))
    b = min(ncell_per_proc, mesh.ncell // k)
    d = tempfile.mkdtemp(prefix="oracle_blocks_")
    try:
        np.save(os.path.join(d, "cmap.npy"), np.ascontiguousarray(cmap))
        np.save(os.path.join(d, "cv.npy"), np.ascontiguousarray(mesh.cell_vertex))
        np.save(os.path.join(d, "coords.npy"), np.ascontiguousarray(mesh.coords))
        np.save(os.path.join(d, "x.npy"), np.ascontiguousarray(x))
        with open(os.path.join(d, "meta.json"), "w") as fh:
            json.dump({"nn": int(nn), "dim": int(wl["dim"]), "p": int(wl["p"])}, fh)
        with mp.get_context("spawn").Pool(k) as pool:
            warm = min(b, 256)  # imports and library load in every process, outside the timing
            pool.map_async(_oracle_block_worker, [(d, i * warm, (i + 1) * warm) for i in range(k)],
                           chunksize=1).get(timeout_s)
            t0 = time.perf_counter()
            secs = pool.map_async(_oracle_block_worker, [(d, i * b, (i + 1) * b) for i in range(k)],
                                  chunksize=1).get(timeout_s)
            wall = time.perf_counter() - t0
    finally:
        shutil.rmtree(d, ignore_errors=True)
    return {"value": k * b / wall, "unit": "cells/s", "cores": k, "kind": "oracle",
            "sample": f"{k} processes (one per host core), each on its own block of {b} cells of the workload mesh "
                      f"(sparsity + assembly + action per block, the blocks' matrices not merged), {wall:.1f} s wall, "
                      f"{max(secs):.1f} s for the slowest block"}


def ref_budget_s(args):
    """Seconds of oracle work per reference step so that warm-up plus timed steps take about two
    minutes in total (never more than --ref-seconds per step)."""
    return min(args.ref_seconds, max(0.05, 120.0 / (args.steps + args.warmup)))


def run_reference(args, wl):
    import oracle
    oracle.build()
    args.ref_seconds = ref_budget_s(args)
    if wl.get("sweep"):
        wl = dict(wl, n=wl["ns"][-1])
    if wl.get("cg"):
        import oracle as O
        reqs = make_serve_inputs(dict(WORKLOADS["serve"]))
        r = max(reqs, key=lambda q: q["nn"] * (q["p"] ** 2))
        rp, ci = O.sparsity(r["cmap"], r["cmap"], r["nn"], r["nn"])
        v, _ = O.assemble_mat(2, r["p"], O.LAPLACE, r["cmap"], r["mesh"].coords, r["mesh"].cell_vertex, rp, ci)
        b, _ = O.assemble_vec(2, r["p"], r["p"], r["cmap"], r["nn"], r["mesh"].coords, r["mesh"].cell_vertex, r["f"],
                              r["cmap"])
        v, b = O.dirichlet_apply(rp, ci, v, b, r["bc"])
        t0 = time.perf_counter()
        O.cg_jacobi(rp, ci, v, b, rtol=1e-30, maxit=5)
        per = max((time.perf_counter() - t0) / 5, 1e-6)
        iters = max(5, int(args.ref_seconds / per))
        res = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            O.cg_jacobi(rp, ci, v, b, rtol=1e-30, maxit=iters)
            res.append(time.perf_counter() - t0)
        vv = iters * len(res) / sum(res)
        return {"impl": "reference", "metric": "CG iterations/s (one system alone)", "value": vv,
                "unit": "iterations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 / vv, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["name"], "reference": "CPU FP64 oracle CG (plain C)"},
                "cpu_baseline": {"value": vv, "unit": "iterations/s", "cores": 1, "kind": "oracle",
                                 "sample": f"{iters} oracle CG iterations per step"},
                "e2e": {"value": vv, "unit": "iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if wl.get("wave"):
        mesh, cmap, nn, _ = make_inputs(wl)
        from paper_1501_01809_gb300 import meshgen as mg
        inputs = (mesh, cmap, nn, mg.face_nodes(mesh, 1, 1, 0))
        res = [wave_cpu_sample(wl, inputs, args.ref_seconds) for _ in range(args.steps)]
        v = sum(c for c, _ in res) / sum(t for _, t in res)
        ms = 1e3 * sum(t for _, t in res) / max(1, sum(c for c, _ in res) // mesh.ncell)
        return {"impl": "reference", "metric": "cells/s stepped (explicit wave: action + lumped-mass updates per "
                                               "time step)", "value": v, "unit": "cells/s", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["name"], "reference": "CPU FP64 oracle (plain C), bounded time per step"},
                "cpu_baseline": {"value": v, "unit": "cells/s", "cores": 1, "kind": "oracle",
                                 "sample": f"oracle time steps of the workload mesh, about {args.ref_seconds} s each"},
                "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if wl.get("serve"):
        reqs = make_serve_inputs(wl)
        res = [serve_cpu_sample(reqs, args.ref_seconds) for _ in range(args.steps)]
        v = sum(c for c, _ in res) / sum(t for _, t in res)
        ms = 1e3 * sum(t for _, t in res) / max(1, sum(c for c, _ in res))
        return {"impl": "reference", "metric": METRIC_SERVE, "value": v, "unit": "solves/s", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["name"], "reference": "CPU FP64 oracle (plain C), requests in order, "
                                                                "bounded time per step"},
                "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                 "sample": f"requests with n <= {SERVE_CPU_MAX_N} in arrival order, about "
                                           f"{args.ref_seconds} s per step"},
                "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if "count" in wl:
        meshes = make_batch_inputs(wl)
        batch_cpu_sample(meshes[:4], 1.0)
        res = [batch_cpu_sample(meshes, args.ref_seconds) for _ in range(args.steps)]
        v = sum(c for c, _ in res) / sum(t for _, t in res)
        ms = 1e3 * sum(t for _, t in res) / len(res)
        return {"impl": "reference", "metric": METRIC_BATCH, "value": v, "unit": "cells/s", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["name"], "reference": "CPU FP64 oracle (plain C), first meshes of the "
                                                                "batch per step (bounded time)"},
                "cpu_baseline": {"value": v, "unit": "cells/s", "cores": 1, "kind": "oracle",
                                 "sample": f"first meshes of the batch, about {args.ref_seconds} s per step"},
                "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    inputs = make_inputs(wl)
    probe = max(_oracle_sample(wl, inputs, 512) / 512, 1e-7)
    ns = int(max(256, min(args.ref_cells, ref_budget_s(args) / probe)))
    for _ in range(args.warmup):
        _oracle_sample(wl, inputs, ns)
    times = [_oracle_sample(wl, inputs, ns) for _ in range(args.steps)]
    ms = 1e3 * sum(times) / len(times)
    v = ns / (ms / 1e3)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "cells/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "reference": "CPU FP64 oracle (plain C), bounded sample per step"},
            "cpu_baseline": {"value": v, "unit": "cells/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {ns} cells of the workload mesh per step"},
            "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def emit(out, args):
    """Prints the run's one JSON line; with --log also appends it, with the time and the command
    line, to a JSONL file (one record per run)."""
    line = json.dumps(out)
    print(line)
    if getattr(args, "log", None):
        rec = dict(out, logged_at=time.strftime("%Y-%m-%dT%H:%M:%S%z"), argv=sys.argv[1:])
        with open(args.log, "a") as fh:
            fh.write(json.dumps(rec) + "\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="p2-3d", choices=sorted(WORKLOADS))
    ap.add_argument("--strategy", default="push", choices=["push", "pull", "auto"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "f32x2"],
                    help="element arithmetic: fp64 (the step of record) or f32x2 (double-float element tensors)")
    ap.add_argument("--no-f32x2", action="store_true", help="skip the labelled double-float extra of the fp64 step")
    ap.add_argument("--cpu-cells", type=int, default=65536, help="oracle sample size for cpu_baseline")
    ap.add_argument("--ref-cells", type=int, default=8192, help="oracle sample per step for --impl reference")
    ap.add_argument("--ref-seconds", type=float, default=2.0, help="oracle seconds per step (batch workload)")
    ap.add_argument("--n", type=int, default=0, help="override the mesh size (profiling on a smaller case)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fuse", default="on", choices=["on", "off"],
                    help="FP64 push step: assembly and action in one pass (on) or as separate kernels (off)")
    ap.add_argument("--copy-streams", type=int, default=1,
                    help="streams per copy direction in the end-to-end leg (each direction's bytes cut evenly)")
    ap.add_argument("--graph", default="auto", choices=["auto", "on", "off"],
                    help="p2-3d/p1-2d: replay the step as one captured CUDA graph (auto: push strategy on one "
                         "stream)")
    ap.add_argument("--overlap", default="off", choices=["off", "on", "hi", "asm", "asm-hi"],
                    help="p2-3d push: Mat zero and action on a second stream beside the sparsity rebuild "
                         "(hi: that stream at high priority); asm: the action on a second stream beside the "
                         "Mat zero and assembly, after the rebuild")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stored", action="store_true", help="skip the stored-matrix action measurement")
    ap.add_argument("--log", default=None, help="also append the JSON line to this JSONL file")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    wl = dict(WORKLOADS[args.workload])
    if args.n and "count" in wl:
        wl["count"] = args.n
        wl["name"] = f"{wl['name']} [count overridden to {args.n}]"
    elif args.n:
        wl["n"] = args.n
        wl["name"] = f"{wl['name']} [n overridden to {args.n}]"
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            emit(run_reference(args, wl), args)
        return
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        td.init_process_group("nccl")
    if wl.get("sweep"):
        out = run_p1_sweep(args, wl, rank, world)
        if rank == 0:
            emit(out, args)
        return
    if wl.get("p4"):
        out = run_p4(args, wl, rank, world)
        if rank == 0:
            emit(out, args)
        return
    if wl.get("cg"):
        out = run_cg(args, wl, rank, world)
        if rank == 0:
            emit(out, args)
        return
    if wl.get("wave"):
        out, winputs = run_wave(args, wl, rank, world)
        if rank == 0:
            if world == 1 and not args.no_cpu_baseline:
                import oracle
                oracle.build()
                cells, dt_s = wave_cpu_sample(wl, winputs, 15.0)
                out["cpu_baseline"] = {"value": cells / dt_s, "unit": "cells/s", "cores": 1, "kind": "oracle",
                                       "sample": f"{cells // winputs[0].ncell} oracle time steps of the workload "
                                                 f"mesh in one call (its lumped-mass assembly included), "
                                                 f"{dt_s:.1f} s on 1 host core"}
            emit(out, args)
        return
    if wl.get("serve"):
        out, reqs = run_serve(args, wl, rank, world)
    elif "count" in wl:
        out, meshes = run_batch(args, wl, rank, world)
    else:
        out, inputs = run_ours(args, wl, rank, world)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline and wl.get("serve"):
            import oracle
            oracle.build()
            done, dt = serve_cpu_sample(reqs, 15.0)
            out["cpu_baseline"] = {"value": done / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                   "sample": f"{done} solves of the requests with n <= {SERVE_CPU_MAX_N}, in arrival "
                                             f"order and repeated (sparsity, assembly, elimination, CG), {dt:.1f} s "
                                             f"on 1 host core; larger requests are left out of the sample"}
        elif world == 1 and not args.no_cpu_baseline and "count" in wl:
            import oracle
            oracle.build()
            batch_cpu_sample(meshes[:4], 1.0)
            cells, dt = batch_cpu_sample(meshes, 15.0)
            out["cpu_baseline"] = {"value": cells / dt, "unit": "cells/s", "cores": 1, "kind": "oracle",
                                   "sample": f"first meshes of the batch ({cells} cells: sparsity + CSR + RHS), "
                                             f"{dt:.1f} s on 1 host core"}
        elif world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(wl, inputs, min(args.cpu_cells, inputs[0].ncell))
            try:  # the same oracle on all host cores: reported beside the one-core figure
                out["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(wl, inputs, min(args.cpu_cells,
                                                                                          inputs[0].ncell))
            except Exception as exc:  # a failed side measurement must not lose the bench line
                out["cpu_baseline"]["all_cores"] = {"error": f"{type(exc).__name__}: {exc}"}
        emit(out, args)
    if world > 1:
        import torch.distributed as td
        td.barrier()
        td.destroy_process_group()


if __name__ == "__main__":
    main()
