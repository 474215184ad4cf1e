"""Throughput of the adaptive 3D Euler ADER-DG step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload euler3d-n5-amr | euler3d-n7-amr | euler2d-n3-vortex]
                    [--precision fp64|fp32]

Default workload: 3D compressible Euler, order N = 5 (6^3 Gauss-Legendre nodes
per cell, 5 variables), spacetree base 27^3 on the periodic unit cube, 3:1
refinement to 2 extra levels inside a ball of radius 0.15 around a Gaussian
density bubble (amplitude 0.2 on rho = 1, p = 1, v = (1, 1, 1)), 2:1 balanced,
remeshing every 10 steps as the ball moves with the flow, skeleton/enclave
streams, FP64.  One bench step = one full ADER-DG time step (predictor,
prolongation, Riemann, restriction, corrector, CFL reduction; the remesh of
every 10th step is inside the timed region).

Metric: DoF-updates/s = sum over cells of m n^3, times steps, over time.
Multi-GPU runs (torchrun) partition the one mesh along its depth-first cell
order (strong scaling): each rank steps its sub-domain and exchanges the
partition-face data every step; the value sums all ranks' owned DoF-updates
over the slowest rank's time.
"""
import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "3D Euler ADER-DG DoF-updates/s on 1 GB300; mixed vs FP64 at same L2 err"
FP64_PEAK_TFLOPS = 1.25   # GB300 FP64 rate (nominal); a pure DFMA loop measured 1.20
FP32_PEAK_TFLOPS = 2 * 152 * 128 * 2.07e9 / 1e12   # 128 FP32 lanes/SM, FMA = 2 flops


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


_PEAKS = _measured_peaks()
# measured copy bandwidth (fallback 6.8 TB/s) and cuBLAS bf16 burst rate;
# dense TF32 on the tensor cores is half the bf16 rate
HBM_PEAK_GBS = float(_PEAKS.get("hbm_gbs", 6800.0))
TF32_PEAK_TFLOPS = float(_PEAKS.get("bf16_tflops", 1900.0)) / 2

# DRAM bytes (read + write) per cell of one predictor launch, from the ncu
# captures summarised in profiles/ for the current kernel versions (small
# case of the same kernel, scaled by cells; per-cell traffic is size
# independent).  A kernel change invalidates its entry.
NCU_TRAFFIC_PER_CELL = {
    "predict_kernel<3,5,Euler,double>": (175.51e6 + 458.56e6) / 19683,
}

WORKLOADS = {
    "euler3d-n5-amr": dict(dim=3, order=5, base=27, max_level=2, radius=0.15, remesh_every=10,
                           init="bubble"),
    "euler3d-n5-base27": dict(dim=3, order=5, base=27, max_level=0, radius=0.0, remesh_every=0,
                              init="bubble"),
    "euler3d-n7-amr": dict(dim=3, order=7, base=27, max_level=2, radius=0.15, remesh_every=10,
                           init="bubble"),
    "euler2d-n3-vortex": dict(dim=2, order=3, base=27, max_level=0, radius=0.0, remesh_every=0,
                              init="vortex"),
}


def predictor_flops_per_cell(dim, order, iters, m):
    """Algorithmic flops of the fused predictor per cell (FMA = 2).

    c_f: one Euler flux evaluation in all dim directions (reciprocal, dim
    velocities, kinetic energy, pressure, E + p, dim(dim+1)/2 momentum
    products, dim pressure terms, dim energy fluxes).  Per node: the first
    Picard iteration needs one time slice (its guess is constant in time);
    each later iteration n slices of flux, divergence (dim m dot products of
    length n) and time mixing (n m FMAs); then n flux evaluations with the
    time averages, the volume term, and the face extrapolation per face node."""
    n = order + 1
    NS = n ** dim
    NF = n ** (dim - 1)
    c_f = 1 + dim + 2 * dim + 3 + 1 + dim * (dim + 1) // 2 + dim + dim
    slice_cost = c_f + dim * m * 2 * n + 2 * n * m
    per_node = slice_cost + (iters - 1) * n * slice_cost
    per_node += n * (c_f + 2 * m * (1 + dim)) + dim * m * 2 * n + 2 * m
    return NS * per_node + 2 * dim * NF * 2 * m * 2 * n


def predictor_bytes_per_cell(dim, order, m):
    """Algorithmic HBM bytes of the fused predictor per cell: read u, write u*
    and the 2d face blocks (Q-bar and F-bar)."""
    n = order + 1
    return 8 * (2 * m * n ** dim + 2 * 2 * dim * m * n ** (dim - 1))


def euler_speed_flops(dim):
    """Flops of one Euler wave-speed estimate |v_d| + sqrt(gamma p / rho),
    division and square root counted as one flop each: reciprocal of rho,
    dim velocities, kinetic energy (2 dim), pressure (2), sound speed (3)."""
    return 1 + dim + 2 * dim + 2 + 3 + 1


def fp64_step_flops_per_cell(dim, order, m):
    """Algorithmic FP64 flops per cell of one step outside the predictor:
    Rusanov on the cell's dim faces (two wave speeds and 3 m flops per face
    node), the corrector lifting (2 dim FMAs and one FMA per node and
    variable) and the CFL rate (dim wave speeds per node)."""
    n = order + 1
    NS, NF = n ** dim, n ** (dim - 1)
    riemann = dim * NF * (2 * euler_speed_flops(dim) + 3 * m)
    corrector = NS * m * (4 * dim + 2)
    rate = NS * (dim * euler_speed_flops(dim) + dim)
    return riemann + corrector + rate


def step_bytes_per_cell(dim, order, m):
    """Minimum HBM bytes per cell of one step with the predictor fused with
    the volume term: u read by the predictor, u* written and re-read, u
    written by the corrector (4 m n^d doubles), and the face data: Q-bar and
    F-bar written and read by the Riemann solves, F* written and read by the
    corrector (11 m n^(d-1) doubles per face slot pair, d slot pairs)."""
    n = order + 1
    return 8 * (4 * m * n ** dim + 11 * dim * m * n ** (dim - 1))


def contraction_tc_flops_per_cell(dim, order, iters, m):
    """Tensor-core flops per cell of the tcgen05 predictor: per Picard slice
    and direction the m n^(d-1) lines padded to M = 128 tiles, times N = 16
    columns and K = 8 (the coordinate along the line, padded), 2 per MAC."""
    n = order + 1
    rows = m * n ** (dim - 1)
    tiles = (rows + 127) // 128
    slices = 1 + (iters - 1) * n
    return slices * dim * tiles * 128 * 16 * 8 * 2


# FP32 instructions per FP64 flop of the double-float predictor (the
# compensated multiply-add of a contraction term: TwoProduct by FMA 2,
# TwoSum 6, the low-part FMA and add 2, and the renormalisation amortised
# over the sum, about 2).
DF64_FP32_PER_FLOP = 6


def step_roofline(prec, dim, order, m, ncells, step_s):
    """Step-level bound: each term is the algorithmic work of one unit over
    its measured or nominal peak; the binding term is the largest, and frac
    = its time over the measured step time."""
    iters = order + 1
    pred = predictor_flops_per_cell(dim, order, iters, m) * ncells
    terms = {"hbm": step_bytes_per_cell(dim, order, m) * ncells / (HBM_PEAK_GBS * 1e9),
             "fp64_faces_corrector": fp64_step_flops_per_cell(dim, order, m) * ncells /
             (FP64_PEAK_TFLOPS * 1e12)}
    if prec == "fp64":
        terms["fp64_faces_corrector"] += pred / (FP64_PEAK_TFLOPS * 1e12)
        terms = {"hbm": terms["hbm"], "fp64_alu": terms["fp64_faces_corrector"]}
    elif prec == "df64":
        # FP32 instructions over the FP32 instruction rate (half the FMA-counted peak)
        terms["fp32_predictor"] = DF64_FP32_PER_FLOP * pred / (FP32_PEAK_TFLOPS * 1e12 / 2)
    elif prec == "fp32":
        terms["fp32_predictor"] = pred / (FP32_PEAK_TFLOPS * 1e12)
    else:
        tc = contraction_tc_flops_per_cell(dim, order, iters, m) * ncells
        products = 1 if prec == "tf32" else 3
        terms["tensor_contractions"] = products * tc / (TF32_PEAK_TFLOPS * 1e12)
        div = (1 + (iters - 1) * (order + 1)) * (order + 1) ** dim * dim * m * 2 * (order + 1)
        terms["fp32_predictor_rest"] = (pred - div * ncells) / (FP32_PEAK_TFLOPS * 1e12)
    bound = max(terms, key=terms.get)
    return {"bound": bound, "bound_ms": terms[bound] * 1e3, "step_ms": step_s * 1e3,
            "frac": terms[bound] / step_s, "terms_ms": {k: v * 1e3 for k, v in terms.items()},
            "peaks": {"fp64_tflops": FP64_PEAK_TFLOPS, "fp32_tflops": FP32_PEAK_TFLOPS,
                      "tf32_tflops": TF32_PEAK_TFLOPS, "hbm_gbs": HBM_PEAK_GBS}}


def bind_near_gpu(torch, index):
    """Pin this process to the CPUs of the GPU's NUMA node (sysfs), so that
    pinned host buffers are first touched, hence allocated, next to the GPU.
    Best effort: returns the CPU list used, or None."""
    try:
        p = torch.cuda.get_device_properties(index)
        bus = "%04x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        text = open(f"/sys/bus/pci/devices/{bus}/local_cpulist").read().strip()
        cpus = set()
        for part in text.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        cpus &= os.sched_getaffinity(0)
        if cpus:
            os.sched_setaffinity(0, cpus)
            return sorted(cpus)
    except Exception:
        return None
    return None


def reduce_over_ranks(torch, seconds, units, device):
    """Whole-job figures of independent replicas: the slowest rank's time and
    the units all ranks processed (any process-group backend)."""
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ader_clocks_{os.getpid()}_{index}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            lines = fh.read().splitlines()
        try:
            os.remove(self.path)
        except OSError:
            pass
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), reasons=parts[4:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        seen = set()
        for r in rows:
            for nm, v in zip(names[1:], r["reasons"][1:]):
                if v.lower() in ("active", "1", "yes"):
                    seen.add(nm)
        return {"sm_mhz": float(np.median([r["sm"] for r in rows])),
                "sm_max_mhz": max(r["smax"] for r in rows), "reasons": sorted(seen),
                "samples": len(rows)}


_U0_CACHE = {}


PIPELINE_CHUNKS = 0   # ader_step enclave chunks (0 = the library default)
PIPELINE_CTAS = 0     # CTAs per SM of the overlapping face/corrector kernels (0 = default)


def build_problem(wl, precision, device):
    from paper_1806_07984_gb300 import Solver
    dim, order = wl["dim"], wl["order"]
    s = Solver(dim, order, "euler", base=(wl["base"],) * 3, max_level=wl["max_level"],
               cfl=workloads.ADER_CFL[order], precision=precision, device=device,
               pipeline_chunks=PIPELINE_CHUNKS, pipeline_ctas=PIPELINE_CTAS)
    center = workloads.sphere_center(0.0)[:dim]
    for _ in range(wl["max_level"]):
        s.remesh(s.sphere_flags(center, wl["radius"]))
    if wl["max_level"] > 0:
        s.classify(s.sphere_flags(center, wl["radius"]))
    key = (id(wl), s.ncells)
    if key not in _U0_CACHE:
        X = s.node_coords()
        if wl["init"] == "bubble":
            u = workloads.density_bubble(X)
        else:
            u = workloads.isentropic_vortex(X[0], X[1])
        _U0_CACHE.clear()
        _U0_CACHE[key] = np.ascontiguousarray(np.moveaxis(u, 0, 1))
    return s, _U0_CACHE[key]


def dofs_of(s):
    return s.ncells * s.nvar * s.n ** s.dim


REMESH_LOG = []   # seconds per remesh + reclassification inside run_steps


def run_steps(s, wl, k, t_dev, step_base):
    """k full steps; every remesh_every-th step is followed by a remesh at the
    ball's current position and a reclassification of the skeleton (host
    time of each, after the device finished the steps before it, goes to
    REMESH_LOG)."""
    dofs = 0
    for i in range(k):
        dofs += dofs_of(s)
        t_dev.add_(s.dt)           # the step advances by the dt it reads
        s.step(1)
        j = step_base + i + 1
        if wl["remesh_every"] and j % wl["remesh_every"] == 0:
            t = float(t_dev.item())
            r0 = time.perf_counter()
            center = workloads.sphere_center(t)[:wl["dim"]]
            s.remesh(s.sphere_flags(center, wl["radius"]))
            s.classify(s.sphere_flags(center, wl["radius"]))
            REMESH_LOG.append(time.perf_counter() - r0)
    return dofs


def run_steps_dd(sub, ex, wl, k, t_dev, step_base):
    """run_steps for one rank's sub-domain of a partitioned mesh: the
    exchange of partition-face data inside every step, dt as the minimum
    over ranks, and remeshing with whole-mesh flags plus the migration of the
    cells that change owner (DoF-updates of the owned cells)."""
    from paper_1806_07984_gb300 import domain
    s = sub.solver
    dofs = 0
    for i in range(k):
        dofs += dofs_of(s)
        t_dev.add_(s.dt)
        domain.step_dist(sub, ex, 1)
        j = step_base + i + 1
        if wl["remesh_every"] and j % wl["remesh_every"] == 0:
            t = float(t_dev.item())
            r0 = time.perf_counter()
            center = workloads.sphere_center(t)[:wl["dim"]]
            flags = s.sphere_flags(center, wl["radius"])
            domain.remesh_dist(sub, ex, flags)
            s.classify(s.sphere_flags(center, wl["radius"]))
            REMESH_LOG.append(time.perf_counter() - r0)
    return dofs


def l2_error_vs_exact(s, u_dev, t, init="bubble", maxes=None):
    """Per-variable L2 error (GL quadrature) of the state against the exact
    solution at time t (the translated bubble or vortex), relative to the L2
    norm of the exact state; with a list `maxes`, also the per-variable
    nodal max error relative to the exact state's max (appended to it)."""
    import torch
    X = s.node_coords()
    q = workloads.density_bubble(X, t=t) if init == "bubble" else \
        workloads.isentropic_vortex(X[0], X[1], t=t)
    ex = np.ascontiguousarray(np.moveaxis(q, 0, 1))
    del X
    xi = s.nodes()
    w = np.polynomial.legendre.leggauss(s.n)[1] / 2.0
    cells = s.cells()
    vol = np.ones(len(cells))
    for d in range(s.dim):
        vol *= (s.cfg.hi[d] - s.cfg.lo[d]) / (s.cfg.base[d] * 3.0 ** cells[:, 0])
    W = w
    for _ in range(s.dim - 1):
        W = np.multiply.outer(W, w)
    errs, norms = [], []
    got = u_dev.cpu().numpy()
    for v in range(s.nvar):
        e = ((got[:, v] - ex[:, v]) ** 2 * W).reshape(len(cells), -1).sum(axis=1)
        nrm = (ex[:, v] ** 2 * W).reshape(len(cells), -1).sum(axis=1)
        errs.append(float(np.sqrt((e * vol).sum())))
        norms.append(float(np.sqrt((nrm * vol).sum())))
        if maxes is not None:
            maxes.append(float(np.abs(got[:, v] - ex[:, v]).max() / np.abs(ex[:, v]).max()))
    del xi
    return [e / nv for e, nv in zip(errs, norms)], got


VAR_NAMES = {2: ["rho", "rho_u", "rho_v", "E"], 3: ["rho", "rho_u", "rho_v", "rho_w", "E"]}


def precision_sweep(torch, wl, precs, steps, warmup, device, base=None):
    """The same workload with each predictor precision: DoF-updates/s over
    `steps` steps after `warmup` (remeshing included), the speed-up over the
    FP64 step, the L2 error against the exact solution, per-variable relative
    L2 and max error against the FP64 result, the predictor's launch time and
    the step-level roofline.  `base` = (value, state, cells) of an FP64 run
    of the same steps; without it the first entry of precs must be fp64."""
    out = {}
    names = VAR_NAMES[wl["dim"]]
    stream = torch.cuda.current_stream()
    for prec in precs:
        if prec in ("tf32", "tf32x3", "bf16x3") and not (wl["dim"] == 3 and wl["order"] >= 5):
            continue
        sm_, u0m = build_problem(wl, prec, device)
        sm_.set_state(torch.from_numpy(u0m).to(device))
        sm_.compute_dt()
        t_m = torch.zeros(1, dtype=torch.float64, device=device)
        run_steps(sm_, wl, warmup, t_m, 0)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        dofs_m = run_steps(sm_, wl, steps, t_m, warmup)
        f1.record(stream)
        torch.cuda.synchronize()
        el_m = f0.elapsed_time(f1) / 1e3
        mx_m = []
        err_m, state_m = l2_error_vs_exact(sm_, sm_.get_state(), float(t_m.item()), wl["init"], mx_m)
        value = dofs_m / el_m
        entry = {"value": value, "unit": "DoF-updates/s", "ms_per_step": el_m / steps * 1e3,
                 "l2_rel_err_vs_exact": dict(zip(names, err_m)),
                 "max_rel_err_vs_exact": dict(zip(names, mx_m)), "status": sm_.status()}
        if prec == "fp64" and base is None:
            base = (value, state_m, sm_.cells())
        else:
            entry["speedup_vs_fp64"] = value / base[0]
            if np.array_equal(sm_.cells(), base[2]):
                entry["vs_fp64_per_var"] = {
                    names[v]: {"rel_l2": float(np.linalg.norm(state_m[:, v] - base[1][:, v]) /
                                               np.linalg.norm(base[1][:, v])),
                               "rel_max": float(np.abs(state_m[:, v] - base[1][:, v]).max() /
                                                np.abs(base[1][:, v]).max())}
                    for v in range(sm_.nvar)}
        t_pred = time_predictor(sm_, torch)
        flops = predictor_flops_per_cell(sm_.dim, sm_.order, sm_.order + 1, sm_.nvar) * sm_.ncells
        entry["predictor_launch_ms"] = t_pred * 1e3
        entry["predictor_tflops"] = flops / t_pred / 1e12
        entry["step_roofline"] = step_roofline(prec, sm_.dim, sm_.order, sm_.nvar, sm_.ncells,
                                               el_m / steps)
        out[prec] = entry
        del state_m
        sm_.close()
    return out, base


def batch_state(sides, orders, specs):
    """Concatenated vortex states of the batch in the library layout."""
    parts = []
    for side, order, sp in zip(sides, orders, specs):
        n = order + 1
        xi = (np.polynomial.legendre.leggauss(n)[0] + 1.0) / 2.0
        c = np.arange(side * side)
        cx, cy = (c % side).astype(np.float64), (c // side).astype(np.float64)
        X = (cx[:, None, None] + xi[None, None, :]) / side + 0 * xi[None, :, None]
        Y = (cy[:, None, None] + xi[None, :, None]) / side + 0 * xi[None, None, :]
        q = workloads.isentropic_vortex(X, Y, center=sp["center"], eps=sp["eps"])
        parts.append(np.ascontiguousarray(np.moveaxis(q, 0, 1)).ravel())
    return np.concatenate(parts)


def run_batched(torch, precision, steps, warmup, count=512):
    """512 seeded 2D Euler instances (sides 9..81, orders 3..7, random
    vortices) advanced by one CUDA-graph launch of persistent phase kernels."""
    from paper_1806_07984_gb300 import ader as A
    specs = workloads.batch_instances(count, seed=0)
    sides = [sp["side"] for sp in specs]
    orders = [sp["order"] for sp in specs]
    cfg = A.ader_batch_config()
    cfg.dim, cfg.pde, cfg.gamma, cfg.picard_iters = 2, A.ADER_EULER, workloads.GAMMA, 0
    cfg.prec = A.ADER_FP64 if precision == "fp64" else A.ADER_FP32
    b = A.ader_batch_init(cfg, sides, orders, [workloads.ADER_CFL[o] for o in orders])
    u = torch.from_numpy(batch_state(sides, orders, specs)).cuda()
    A.ader_batch_set_state(b, u.data_ptr(), True)
    A.ader_batch_compute_dt(b)
    bps, tile, tune_ms = A.ader_batch_tune(b)
    A.ader_batch_run(b, warmup)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = A.ader_batch_launch_count(b)
    e0.record(st)
    A.ader_batch_run(b, steps, st.cuda_stream)
    e1.record(st)
    torch.cuda.synchronize()
    el = e0.elapsed_time(e1) / 1e3
    launches = A.ader_batch_launch_count(b) - l0
    status = A.ader_batch_status_word(b)
    dofs = sum(s * s * 4 * (o + 1) ** 2 for s, o in zip(sides, orders))
    flops = sum(predictor_flops_per_cell(2, o, o + 1, 4) * s * s for s, o in zip(sides, orders))
    peak = FP64_PEAK_TFLOPS if precision == "fp64" else FP32_PEAK_TFLOPS
    achieved = flops * steps / el / 1e12
    A.ader_batch_destroy(b)
    return {"workload": f"{count} 2D Euler instances, sides 9..81, orders 3..7, seed 0",
            "precision": precision, "value": dofs * steps / el, "unit": "DoF-updates/s",
            "steps": steps, "ms_per_step": el / steps * 1e3, "dofs": dofs,
            "cells": sum(s * s for s in sides), "graph_launches": 1,
            "kernel_launches": launches, "tuned": {"ctas_per_sm": bps, "tile": tile,
                                                   "step_ms": tune_ms}, "status": status,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "note": "predictor flops of every instance per step over the whole step's "
                                 "time (faces and corrector included)"}}


def run_dd_virtual(torch, nranks=4, steps=5, warmup=2):
    """The bench mesh split into `nranks` sub-domains of the SFC partition on
    one GPU (virtual ranks, device copies between their exchange buffers),
    stepped together, against the same steps of the unpartitioned context
    with the enclave pipeline off (the sub-domains run one chunk each): the
    cost of the ghost faces, the halo packing and the exchange."""
    from paper_1806_07984_gb300 import domain
    global PIPELINE_CHUNKS
    wl = WORKLOADS["euler3d-n5-amr"]
    dev = torch.device("cuda", 0)
    saved, PIPELINE_CHUNKS = PIPELINE_CHUNKS, 1
    try:
        ref, u0 = build_problem(wl, "fp64", dev)
        subs = []
        for r in range(nranks):
            s, _ = build_problem(wl, "fp64", dev)
            s.set_state(u0)
            s.compute_dt()
            subs.append(domain.SubDomain(s, nranks, r))
    finally:
        PIPELINE_CHUNKS = saved
    ref.set_state(u0)
    ref.compute_dt()
    ex = domain.LocalExchange(subs)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ref.step(warmup)
    torch.cuda.synchronize()
    e0.record(st)
    ref.step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    t_ref = e0.elapsed_time(e1) / 1e3
    domain.step_local(subs, ex, warmup)
    torch.cuda.synchronize()
    e0.record(st)
    domain.step_local(subs, ex, steps)
    e1.record(st)
    torch.cuda.synchronize()
    t_dd = e0.elapsed_time(e1) / 1e3
    dofs = dofs_of(ref) * steps
    info = [s.info() for s in subs]
    out = {"workload": f"3D Euler N=5 bench mesh ({ref.ncells} cells), {nranks} sub-domains on one GPU, "
                       f"{steps} steps after {warmup}",
           "value": dofs / t_dd, "unit": "DoF-updates/s", "ms_per_step": t_dd / steps * 1e3,
           "unpartitioned_ms_per_step": t_ref / steps * 1e3, "overhead": t_dd / t_ref - 1.0,
           "owned_cells": [i[4] for i in info], "ghost_cells": [i[5] for i in info],
           "halo_bytes_per_step": sum(s.halo_bytes() for s in subs),
           "status": max(s.solver.status() for s in subs)}
    for s in subs:
        s.solver.close()
    ref.close()
    return out


def run_shifted(torch, precs=("fp64", "fp32", "df64"), steps=6, warmup=2):
    """Global time stepping with a prescribed dt by the shifted task graph
    (ader_step_fixed_dt: the corrector of step k runs as the prologue of the
    predictor of step k + 1, nsteps + 1 cell passes per call) against
    ader_step (CFL time step from every corrector, enclave pipeline, CUDA
    graph) on the bench mesh, both over `steps` steps in one call."""
    wl = WORKLOADS["euler3d-n5-amr"]
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream()
    out = {"workload": "3D Euler N=5 bench mesh, %d steps in one call after %d" % (steps, warmup)}
    for prec in precs:
        s, u0 = build_problem(wl, prec, dev)
        s.set_state(torch.from_numpy(u0).to(dev))
        s.compute_dt()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        s.step(warmup)
        torch.cuda.synchronize()
        ev[0].record(st)
        s.step(steps)
        ev[1].record(st)
        dt_next = torch.zeros(1, dtype=torch.float64, device=dev)
        s.step_fixed_dt(warmup, dt_next)        # dt: the last CFL step of the loop above
        torch.cuda.synchronize()
        ev[2].record(st)
        s.step_fixed_dt(steps, dt_next)
        ev[3].record(st)
        torch.cuda.synchronize()
        t_step = ev[0].elapsed_time(ev[1]) / steps
        t_fix = ev[2].elapsed_time(ev[3]) / steps
        dofs = dofs_of(s)
        out[prec] = {"value": dofs / (t_fix / 1e3), "unit": "DoF-updates/s",
                     "ms_per_step": t_fix, "ader_step_ms_per_step": t_step,
                     "speedup_vs_ader_step": t_step / t_fix, "status": s.status()}
        s.close()
    return out


def run_adjoint(torch, predictor="picard"):
    """3D linear acoustics N=4 on 27^3 (FP64; Picard with 13 iterations or the
    Cauchy-Kowalevski predictor): one loss and gradient with respect to the
    initial state over 50 steps, 64 receivers, checkpoints every 10 steps
    (forward + recomputation + adjoint sweep)."""
    from paper_1806_07984_gb300 import Solver, adjoint as adj, ader as A
    order = 4
    s = Solver(3, order, "acoustics", base=(27, 27, 27), cfl=workloads.ADER_CFL[order],
               picard_iters=3 * order + 1, predictor=predictor)
    X = s.node_coords()
    u0 = torch.from_numpy(np.ascontiguousarray(
        np.moveaxis(workloads.acoustic_pulses(X, seed=1), 0, 1))).cuda()
    uobs = torch.from_numpy(np.ascontiguousarray(
        np.moveaxis(workloads.acoustic_pulses(X, seed=3), 0, 1))).cuda()
    del X
    s.set_state(u0)
    s.compute_dt()
    dt = s.dt.clone()
    rec = adj.Receivers(s, workloads.acoustic_receivers(64, seed=2))
    nsteps = 50
    p_obs, _ = adj.forward_run(s, uobs, dt, rec, nsteps)
    loss_fn = adj.AcousticMisfit.make(s, dt, rec, p_obs, nsteps, every=10)
    w = u0.clone().requires_grad_(True)     # untimed warm-up of the autograd path
    loss_fn(w).backward()
    del w
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    u = u0.clone().requires_grad_(True)
    e0.record(st)
    loss = loss_fn(u)
    e1.record(st)
    loss.backward()
    e2.record(st)
    torch.cuda.synchronize()
    t_fwd = e0.elapsed_time(e1) / 1e3
    t_bwd = e1.elapsed_time(e2) / 1e3
    # one adjoint step kernel sequence, timed alone
    lam = torch.randn_like(u0)
    out = torch.empty_like(u0)
    A.ader_adjoint_step(s.ctx, lam, out, dt)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(5):
        A.ader_adjoint_step(s.ctx, lam, out, dt)
    e1.record(st)
    torch.cuda.synchronize()
    t_adj = e0.elapsed_time(e1) / 5e3
    dofs = s.ncells * s.nvar * s.n ** 3
    s.close()
    return {"workload": "3D acoustics N=4, 27^3 periodic, 50 steps, 64 receivers, checkpoints every 10",
            "predictor": predictor, "loss": float(loss.detach()), "grad_norm": float(u.grad.norm()),
            "forward_s": t_fwd, "backward_s": t_bwd, "gradient_s": t_fwd + t_bwd,
            "adjoint_step_ms": t_adj * 1e3, "adjoint_dof_updates_per_s": dofs / t_adj,
            "dofs": dofs}


def run_limiter(torch, dim=2, order=3, base=729, steps=10, warmup=2):
    """Circular explosion (a density and pressure jump, smoothed over half a
    cell) on a uniform periodic grid with the a posteriori subcell FV limiter;
    DoF-updates/s with and without the limiter on the same run."""
    from paper_1806_07984_gb300 import Solver
    out = {}
    for lim in (True, False):
        s = Solver(dim, order, "euler", base=(base,) * 3, cfl=workloads.ADER_CFL[order], limiter=lim)
        X = s.node_coords()
        u0 = np.ascontiguousarray(np.moveaxis(
            workloads.circular_explosion(X, width=0.5 / base), 0, 1))
        del X
        s.set_state(torch.from_numpy(u0).cuda())
        s.compute_dt()
        s.step(warmup)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        dofs = s.ncells * s.nvar * s.n ** dim
        rec = {"value": dofs * steps / sec, "unit": "DoF-updates/s", "ms_per_step": sec / steps * 1e3,
               "status": s.status()}
        if lim:
            flags, nlim = s.limiter_flags()
            rec["limited_cells_last_step"] = int(nlim)
            rec["limited_fraction"] = nlim / s.ncells
            rec["flux_replaced_cells"] = int(((flags & 2) != 0).sum())
        out["limiter" if lim else "no_limiter"] = rec
        s.close()
    out["workload"] = (f"{dim}D Euler N={order}, {base}^{dim} periodic, circular explosion "
                       f"(rho 1/0.125, p 1/0.1, r=0.25), {steps} steps after {warmup}")
    out["overhead"] = out["no_limiter"]["value"] / out["limiter"]["value"]
    return out


def ck_flops_per_cell(dim, order):
    """Algorithmic flops of the Cauchy-Kowalevski predictor per cell (linear
    acoustics, FMA = 2).  Per node: N time derivatives, each the derivatives
    of the two nonzero flux components of every direction (2n each) and one
    Taylor term per variable (2m); then the volume term (two nonzero
    components per direction, 2n + 2 each) and u* = u + dt vol (2m).  Per face
    node: Q-bar (m variables) and the two nonzero components of F-bar
    extrapolated along the normal (2n each)."""
    n, m = order + 1, dim + 1
    NS, NF = n ** dim, n ** (dim - 1)
    per_node = order * (dim * 2 * 2 * n + 2 * m) + dim * 2 * (2 * n + 2) + 2 * m
    return NS * per_node + 2 * dim * NF * (m + 2) * 2 * n


def run_ck(torch, order=4, base=54, steps=5, warmup=3):
    """3D linear acoustics N=4 on a uniform periodic base^3 grid (eight seeded
    Gaussian pressure pulses; base 54: the 0.63 GB state exceeds L2): the
    forward step with the Cauchy-Kowalevski predictor against the Picard
    predictor (N + 1 iterations), and the CK predictor kernel against the
    FP64 ALU peak."""
    from paper_1806_07984_gb300 import Solver
    out = {}
    finals = {}
    for pred in ("ck", "picard"):
        s = Solver(3, order, "acoustics", base=(base,) * 3, cfl=workloads.ADER_CFL[order],
                   predictor=pred)
        X = s.node_coords()
        u0 = np.ascontiguousarray(np.moveaxis(workloads.acoustic_pulses(X, seed=1), 0, 1))
        del X
        s.set_state(torch.from_numpy(u0).cuda())
        del u0
        s.compute_dt()
        s.step(warmup)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        dofs = s.ncells * s.nvar * s.n ** 3
        finals[pred] = s.get_state()
        t_pred = time_predictor(s, torch)
        rec = {"value": dofs * steps / sec, "unit": "DoF-updates/s", "ms_per_step": sec / steps * 1e3,
               "predictor_launch_ms": t_pred * 1e3, "status": s.status()}
        if pred == "ck":
            fl = ck_flops_per_cell(3, order) * s.ncells
            achieved = fl / t_pred / 1e12
            rec["roofline"] = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                               "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                               "algorithmic_flops": fl,
                               "algorithmic_bytes": predictor_bytes_per_cell(3, order, s.nvar) * s.ncells}
        out[pred] = rec
        s.close()
    d = finals["ck"] - finals["picard"]
    out["ck_vs_picard_rel_l2"] = float(d.norm() / finals["picard"].norm())
    del finals, d
    out["workload"] = (f"3D acoustics N={order}, {base}^3 periodic, 8 Gaussian pulses (seed 1), "
                       f"{steps} steps after {warmup}")
    out["speedup"] = out["ck"]["value"] / out["picard"]["value"]
    return out


def indicator_flops_per_cell(dim, order, deriv):
    """Algorithmic flops of the refinement indicator per cell (FMA = 2):
    per node dim first derivatives (2n + 1 each); then either their squares
    (2 each) or the dim (dim + 1) / 2 distinct Hessian entries (2n + 1 each)
    and their weighted squares (2 each)."""
    n = order + 1
    per_node = dim * (2 * n + 1)
    per_node += 2 * dim if deriv == 1 else dim * (dim + 1) // 2 * (2 * n + 3)
    return n ** dim * per_node


def run_indicator(s, torch, reps=5):
    """The solution-based refinement indicator (ader_gradient_indicator on the
    density, first derivatives and Hessian) on the bench mesh: device time per
    launch (CUDA events) against the FP64 ALU peak, and the host-synchronous
    ader_gradient_flags call."""
    from paper_1806_07984_gb300 import ader as A
    st = torch.cuda.current_stream()
    eta = torch.empty(s.ncells, dtype=torch.float64, device=s.device)
    out = {}
    for deriv in (1, 2):
        A.ader_gradient_indicator(s.ctx, 0, eta, st.cuda_stream, deriv)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            A.ader_gradient_indicator(s.ctx, 0, eta, st.cuda_stream, deriv)
        e1.record(st)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        fl = s.ncells * indicator_flops_per_cell(s.dim, s.order, deriv)
        by = s.ncells * (s.n ** s.dim + 1) * 8
        c0 = time.perf_counter()
        s.gradient_flags(0, 1.0, 0.1, deriv)
        t_flags = time.perf_counter() - c0
        out[f"deriv{deriv}"] = {
            "launch_ms": t * 1e3, "cells_per_s": s.ncells / t,
            "roofline": {"bound": "alu", "achieved": fl / t / 1e12, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": fl / t / 1e12 / FP64_PEAK_TFLOPS,
                         "algorithmic_flops": fl, "algorithmic_bytes": by, "hbm_gbs": by / t / 1e9},
            "gradient_flags_call_ms": t_flags * 1e3}
    out["workload"] = "density derivatives on the bench mesh (%d cells)" % s.ncells
    return out


def time_predictor(s, torch, reps=3):
    """Average duration of one ader_predict(ADER_ALL) launch, CUDA events on
    the launching stream."""
    from paper_1806_07984_gb300 import ader as A
    st = torch.cuda.current_stream()
    s.predict(A.ADER_ALL, stream=st)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        s.predict(A.ADER_ALL, stream=st)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def cpu_baseline(wl_name, wl, seconds=15.0, cores=1):
    """Oracle (numpy FP64, one BLAS thread per process) on a bounded sample:
    full oracle steps on the same PDE, order, bubble and refinement rule (ball
    radius) on a base 3^3 mesh; with cores > 1 that many independent processes run at once and
    their throughputs add up."""
    code = r"""
import os, sys, time, json
import numpy as np
sys.path.insert(0, %r)
from oracle import ader, basis, mesh as omesh, pde as opde, step as ostep
import workloads
dim, order, lvl, radius, budget = %d, %d, %d, %r, %r
m = omesh.Mesh(dim, (3,) * dim, lvl)
B = basis.Basis(order)
c = workloads.sphere_center(0.0)[:dim]
u = np.zeros((len(m.cells), 1) + (2,) * dim)
for _ in range(lvl):
    u = m.remesh(u, omesh.sphere_flags(m, c, radius), basis.Basis(1))
X = m.node_coords(B.xi)
u = np.ascontiguousarray(np.moveaxis(workloads.density_bubble(X), 0, 1))
P = opde.Euler(dim)
h = m.cell_widths()
dt = ader.cfl_dt(u, h, P, order, cfl=workloads.ADER_CFL[order])
steps, t0 = 0, time.perf_counter()
while True:
    out = ostep.step(m, u, dt, P, B)
    u, dt = out.u, out.dt_next
    steps += 1
    if time.perf_counter() - t0 > budget:
        break
el = time.perf_counter() - t0
dofs = len(m.cells) * (dim + 2) * (order + 1) ** dim
print(json.dumps(dict(value=dofs * steps / el, cells=len(m.cells), steps=steps, seconds=el)))
""" % (ROOT, wl["dim"], wl["order"], wl["max_level"], wl["radius"], seconds)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    every_cpu = set(range(os.cpu_count() or 1))

    def unbind():   # the bench process may be pinned next to its GPU
        try:
            os.sched_setaffinity(0, every_cpu)
        except OSError:
            pass
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=env, preexec_fn=unbind)
             for _ in range(cores)]
    results = []
    for pr in procs:
        out, err = pr.communicate(timeout=600)
        if pr.returncode != 0:
            return {"error": err[-400:]}
        results.append(json.loads(out.strip().splitlines()[-1]))
    res = results[0]
    what = (f"{res['steps']} oracle steps of the same PDE, order, bubble and refinement ball on a "
            f"base-3^{wl['dim']} mesh with {res['cells']} cells ({res['seconds']:.1f} s, numpy FP64, "
            f"1 BLAS thread)")
    if cores > 1:
        what = f"{cores} concurrent processes, each " + what
    return {"value": sum(r["value"] for r in results), "unit": "DoF-updates/s", "cores": cores,
            "kind": "oracle", "sample": what}


def reference_arm(args, wl_name, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(wl_name, wl, seconds=2.0)
    samples = []
    for _ in range(args.steps):
        r = cpu_baseline(wl_name, wl, seconds=5.0)
        if "value" not in r:
            print(json.dumps({"impl": "reference", "unavailable": r.get("error", "oracle failed")}))
            return
        vals.append(r["value"])
        samples.append(r)
    v = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "DoF-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl_name, "order": wl["order"], "dim": wl["dim"]},
            "cpu_baseline": {"value": v, "unit": "DoF-updates/s", "cores": 1, "kind": "oracle",
                             "sample": samples[0]["sample"]},
            "e2e": {"value": v, "unit": "DoF-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _g(x, digits=3):
    return float(f"{x:.{digits}g}") if isinstance(x, (int, float)) else x


def summarise(line):
    """Compact digest of the line's sections (kept last in the JSON line):
    per precision the speed-up over FP64, the density's L2 error against the
    exact solution and against the FP64 result, and the step's roofline."""
    out = {"fp64": _g(line["value"]), "remesh_ms": line["remesh"]["ms_each"],
           "fp64_step_frac": None}

    def digest(sec):
        d = {}
        for prec, e in sec.items():
            if not isinstance(e, dict) or "value" not in e:
                continue
            ex = e.get("l2_rel_err_vs_exact", {})
            r = e.get("step_roofline", {})
            d[prec] = {"v": _g(e["value"]), "x": _g(e.get("speedup_vs_fp64", 1.0)),
                       "err_rho": _g(ex.get("rho")) if ex else None,
                       "vs64_rho": _g(e.get("vs_fp64_per_var", {}).get("rho", {}).get("rel_l2")),
                       "bound": r.get("bound"), "frac": _g(r.get("frac"))}
        return d
    if line.get("mixed"):
        out["n5"] = digest(line["mixed"])
        out["fp64_step_frac"] = out["n5"].get("fp64", {}).get("frac")
        # per precision, per variable (in `vars` order): relative L2 and max
        # error against the exact solution and against the FP64 result
        names = None
        per = {}
        for prec, e in line["mixed"].items():
            if not isinstance(e, dict) or "l2_rel_err_vs_exact" not in e:
                continue
            names = list(e["l2_rel_err_vs_exact"])
            vs = e.get("vs_fp64_per_var", {})
            per[prec] = {"x": _g(e.get("speedup_vs_fp64", 1.0), 3),
                         "exact_l2": [_g(e["l2_rel_err_vs_exact"][v], 2) for v in names],
                         "exact_max": [_g(e.get("max_rel_err_vs_exact", {}).get(v), 2) for v in names],
                         "vs64_l2": [_g(vs.get(v, {}).get("rel_l2"), 2) for v in names] if vs else None,
                         "vs64_max": [_g(vs.get(v, {}).get("rel_max"), 2) for v in names] if vs else None}
        out["mixed_summary"] = {"vars": names, **per}
    cf = line.get("configs") or {}
    if "euler3d-n7-amr" in cf:
        out["n7"] = digest(cf["euler3d-n7-amr"])
    if "euler2d-n3-vortex" in cf:
        out["vortex_n3"] = digest({"fp64": cf["euler2d-n3-vortex"]})["fp64"]
    if line.get("dd_virtual"):
        out["dd4_overhead"] = _g(line["dd_virtual"]["overhead"])
    if line.get("shifted_fixed_dt"):
        out["shifted_x"] = {p: _g(e["speedup_vs_ader_step"]) for p, e in line["shifted_fixed_dt"].items()
                            if isinstance(e, dict)}
    if "mixed_summary" in out:  # last, so that it ends the line
        out["mixed_summary"] = out.pop("mixed_summary")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="euler3d-n5-amr", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64",
                    choices=["fp64", "fp32", "tf32", "tf32x3", "bf16x3", "df64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mixed", default="df64,fp32,tf32x3,bf16x3,tf32",
                    help="predictor precisions compared with FP64 ('' to skip)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-limiter", action="store_true")
    ap.add_argument("--no-ck", action="store_true")
    ap.add_argument("--section", choices=["ck", "limiter", "adjoint", "batched", "dd", "shifted"],
                    default=None,
                    help="run one side section alone and print its JSON object (no headline)")
    ap.add_argument("--ck-base", type=int, default=54, help="grid of the CK section (base^3)")
    ap.add_argument("--no-indicator", action="store_true")
    ap.add_argument("--no-dd", action="store_true",
                    help="skip the 4-sub-domain partitioned step on one GPU")
    ap.add_argument("--no-shifted", action="store_true",
                    help="skip the prescribed-dt shifted-task-graph steps")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 2D N=3 vortex and 3D N=7 sections")
    ap.add_argument("--pipeline", type=int, default=0,
                    help="enclave chunks per step (0 = library default, 1 = no pipelining)")
    ap.add_argument("--pipeline-ctas", type=int, default=0,
                    help="CTAs per SM of the face/corrector kernels that overlap the predictor")
    args = ap.parse_args()
    global PIPELINE_CHUNKS, PIPELINE_CTAS
    PIPELINE_CHUNKS = args.pipeline
    PIPELINE_CTAS = args.pipeline_ctas
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        reference_arm(args, args.workload, wl)
        return

    import torch
    if args.section:
        torch.cuda.set_device(0)
        out = {"ck": lambda: run_ck(torch, base=args.ck_base),
               "limiter": lambda: {"2d_n3_729": run_limiter(torch, 2, 3, 729),
                                   "3d_n5_27": run_limiter(torch, 3, 5, 27, 5)},
               "adjoint": lambda: {"picard": run_adjoint(torch, "picard"),
                                   "ck": run_adjoint(torch, "ck")},
               "batched": lambda: {"fp64": run_batched(torch, "fp64", 20, 2),
                                   "fp32": run_batched(torch, "fp32", 20, 2)},
               "dd": lambda: run_dd_virtual(torch),
               "shifted": lambda: run_shifted(torch)}[args.section]()
        print(json.dumps({"section": args.section, args.section: out}))
        return
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    near = bind_near_gpu(torch, local)

    s, u0 = build_problem(wl, args.precision, device)
    u_dev = torch.from_numpy(u0).to(device)
    s.set_state(u_dev)
    s.compute_dt()
    # N > 1: one sub-domain of the SFC partition per rank (the whole mesh and
    # state were built on every rank; each keeps its owned cells)
    sub = ex = None
    if world > 1:
        from paper_1806_07984_gb300 import domain
        sub = domain.SubDomain(s, world, rank)
        ex = domain.DistExchange()

    def steps_fn(k, t, base):
        if sub is not None:
            return run_steps_dd(sub, ex, wl, k, t, base)
        return run_steps(s, wl, k, t, base)
    t_dev = torch.zeros(1, dtype=torch.float64, device=device)
    steps_fn(args.warmup, t_dev, 0)
    torch.cuda.synchronize()

    # ---- device-resident timed region -----------------------------------
    stream = torch.cuda.current_stream()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = s.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    REMESH_LOG.clear()
    dofs = steps_fn(args.steps, t_dev, args.warmup)
    remesh_times = list(REMESH_LOG)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = s.launch_count() - launches0
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1e3
    status = s.status()
    if world > 1:
        elapsed, total_dofs = reduce_over_ranks(torch, elapsed, dofs, device)
    else:
        total_dofs = float(dofs)
    value = total_dofs / elapsed

    # ---- dominant kernel: the fused predictor ------------------------------
    t_pred = time_predictor(s, torch)
    iters = s.order + 1
    flops = predictor_flops_per_cell(s.dim, s.order, iters, s.nvar) * s.ncells
    bytes_ = predictor_bytes_per_cell(s.dim, s.order, s.nvar) * s.ncells
    peak = FP64_PEAK_TFLOPS if args.precision == "fp64" else FP32_PEAK_TFLOPS
    achieved = flops / t_pred / 1e12
    if args.precision in ("tf32", "tf32x3", "bf16x3"):
        kname = f"predict_tc_kernel<{s.order},Euler,{args.precision}>"
    else:
        kname = (f"predict_kernel<{s.dim},{s.order},Euler,"
                 f"{'double' if args.precision == 'fp64' else 'float'}>")
    tpc = NCU_TRAFFIC_PER_CELL.get(kname)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": tpc * s.ncells if tpc else None,
                "kernel": kname,
                "launch_ms": t_pred * 1e3, "algorithmic_flops": flops,
                "algorithmic_bytes": bytes_, "hbm_gbs": bytes_ / t_pred / 1e9}

    indicator = run_indicator(s, torch) if not args.no_indicator else None

    # ---- end to end through the public API with host buffers ---------------
    # Every step: H2D of the state from pinned host memory, one step, D2H of
    # the new state into pinned host memory (the step's result).
    from paper_1806_07984_gb300 import ader as A
    e2e_steps = max(2, min(args.steps, 5))
    s2, u02 = build_problem(wl, args.precision, device)
    s2.set_state(u02)
    s2.compute_dt()
    sub2 = None
    if world > 1:
        from paper_1806_07984_gb300 import domain
        sub2 = domain.SubDomain(s2, world, rank)
        ex2 = domain.DistExchange()
    host = s2.get_state().cpu().pin_memory()   # the owned cells (all of them at N = 1)
    del u02

    def steps2(k, t, base):
        if sub2 is not None:
            return run_steps_dd(sub2, ex2, wl, k, t, base)
        return run_steps(s2, wl, k, t, base)
    t_e2e = torch.zeros(1, dtype=torch.float64, device=device)
    steps2(2, t_e2e, 0)                     # untimed warm-up: an eager step, then the step graph
    s2.set_state(host)
    if sub2 is None:
        s2.compute_dt()
    t_e2e.zero_()
    torch.cuda.synchronize()
    c0 = time.perf_counter()
    e2e_dofs = h2d = d2h = 0
    e2e_each = []
    assert not wl["remesh_every"] or e2e_steps < wl["remesh_every"]
    for i in range(e2e_steps):
        t_i = time.perf_counter()
        if sub2 is None:
            # one call: state in from pinned host memory (overlapping the
            # enclave predictor chunks), the step, state out
            e2e_dofs += dofs_of(s2)
            t_e2e.add_(s2.dt)
            A.ader_step_host(s2.ctx, host.data_ptr(), host.data_ptr(), s2.dt.data_ptr(),
                             stream.cuda_stream)
            h2d += host.numel() * 8
            d2h += host.numel() * 8
        else:
            s2.set_state(host)
            h2d += host.numel() * 8
            e2e_dofs += steps2(1, t_e2e, i)
            A.ader_get_state(s2.ctx, host.data_ptr(), False, stream.cuda_stream)
            d2h += host.numel() * 8
        torch.cuda.current_stream().synchronize()
        e2e_each.append(round((time.perf_counter() - t_i) * 1e3, 1))
    torch.cuda.synchronize()
    e2e_time = time.perf_counter() - c0
    e2e_total = float(e2e_dofs)
    if world > 1:
        e2e_time, e2e_total = reduce_over_ranks(torch, e2e_time, e2e_dofs, device)
    e2e = {"value": e2e_total / e2e_time, "unit": "DoF-updates/s",
           "h2d_bytes_per_step": h2d // e2e_steps, "d2h_bytes_per_step": d2h // e2e_steps,
           "steps": e2e_steps, "ms_each": e2e_each, "host_cpus": f"{len(near)} CPUs local to the GPU" if near else "unbound"}
    ncells, dofs_now, order, dim = s2.ncells, dofs_of(s2), s2.order, s2.dim
    halo = sub.halo_bytes() if sub is not None else 0
    ncells_all = A.ader_dd_info(s2.ctx)[2]
    dofs_all = ncells_all * s2.nvar * s2.n ** s2.dim
    s2.close()

    # ---- mixed precision: FP32 / tensor-core predictors on the same workload ----
    mixed = None
    if args.precision == "fp64" and args.mixed and world == 1:
        mx64 = []
        err64, state64 = l2_error_vs_exact(s, s.get_state(), float(t_dev.item()), wl["init"], mx64)
        cells64 = s.cells()
        s.close()
        del u_dev
        names = VAR_NAMES[wl["dim"]]
        mixed, _ = precision_sweep(torch, wl, args.mixed.split(","), args.steps, args.warmup,
                                   device, base=(value, state64, cells64))
        mixed["fp64"] = {"value": value, "l2_rel_err_vs_exact": dict(zip(names, err64)),
                         "max_rel_err_vs_exact": dict(zip(names, mx64)),
                         "step_roofline": step_roofline("fp64", wl["dim"], wl["order"],
                                                        len(names), ncells,
                                                        elapsed / args.steps)}
        mixed["note"] = ("predictor arithmetic: df64 = double-float on the FP32 pipes, fp32 = FP32 "
                         "CUDA cores, tf32/tf32x3/bf16x3 = tcgen05 tensor cores; FP64 state, faces, "
                         "Riemann, corrector and CFL reduction in every mode")
        del state64
    else:
        s.close()
        del u_dev

    # ---- the other workload shapes: config 1 (2D vortex, N=3) and config 3
    # (3D AMR at N=7, FP64 against the mixed predictors) ----------------------
    configs = None
    if not args.no_configs and world == 1 and args.workload == "euler3d-n5-amr":
        configs = {}
        v1, _ = precision_sweep(torch, WORKLOADS["euler2d-n3-vortex"], ["fp64"], 20, 3, device)
        configs["euler2d-n3-vortex"] = dict(v1["fp64"], workload=(
            "2D Euler N=3, 27^2 periodic, isentropic vortex eps=5 on rho=1, v=(1,1), p=1, "
            "20 steps after 3"))
        precs3 = ["fp64"] + [p for p in args.mixed.split(",") if p]
        v3, _ = precision_sweep(torch, WORKLOADS["euler3d-n7-amr"], precs3, 7, 3, device)
        v3["workload"] = ("3D Euler N=7, base 27^3 + 2 levels around the bubble, 7 steps after 3 "
                          "(a remesh inside)")
        configs["euler3d-n7-amr"] = v3

    # ---- batched instances (one CUDA graph per run) --------------------------
    batched = None
    if not args.no_batched and world == 1:
        batched = {"fp64": run_batched(torch, "fp64", 20, 2),
                   "fp32": run_batched(torch, "fp32", 20, 2)}

    adjoint = ({"picard": run_adjoint(torch, "picard"), "ck": run_adjoint(torch, "ck")}
               if (not args.no_adjoint and world == 1) else None)
    limiter = ({"2d_n3_729": run_limiter(torch, 2, 3, 729), "3d_n5_27": run_limiter(torch, 3, 5, 27, 5)}
               if (not args.no_limiter and world == 1) else None)
    ck = run_ck(torch, base=args.ck_base) if (not args.no_ck and world == 1) else None
    dd = run_dd_virtual(torch) if (not args.no_dd and world == 1) else None
    shifted = run_shifted(torch) if (not args.no_shifted and world == 1) else None


    line = {"metric": METRIC, "value": value, "unit": "DoF-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "dim": dim, "order": order,
                       "cells": ncells_all, "dofs": dofs_all, "precision": args.precision,
                       "parallelism": f"sfc{world}" if world > 1 else "single",
                       "halo_bytes_per_step_rank0": halo,
                       "l2": "inputs larger than L2 (state %.1f GB)" % (dofs_all * 8 / 1e9),
                       "remesh_every": wl["remesh_every"],
                       "pipeline_chunks": args.pipeline or 8,
                       "pipeline_ctas_per_sm": args.pipeline_ctas or 4},
            "remesh": {"count_in_timed_steps": len(remesh_times),
                       "ms_each": [round(x * 1e3, 2) for x in remesh_times],
                       "included_in_value": True,
                       "note": "host tree adaptation, list uploads, transfer kernel and skeleton "
                               "reclassification; the paper's timings exclude remeshing"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "status": status,
            "clocks": clk, "mixed": mixed, "batched": batched, "adjoint": adjoint, "limiter": limiter,
            "ck": ck, "indicator": indicator, "configs": configs, "dd_virtual": dd,
            "shifted_fixed_dt": shifted}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, wl)
        line["cpu_baseline_all_cores"] = cpu_baseline(args.workload, wl, seconds=10.0,
                                                      cores=os.cpu_count() or 1)
    line["summary"] = summarise(line)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
