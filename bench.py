#!/usr/bin/env python
"""Benchmark: pair-kernel entries/s of the mixed-precision forward + Jacobian pass on one GB300.

A step is one pass of the whole hot path over the batch: persistent scheduling of all zones,
zone set-up, the (eps, eps', omega, E) quadrature, the spectral contraction and the T / eta_e
tangents (forward rates and the full Jacobian d(j0, chi0, j1, chi1)/d(T, eta_e, Y_e) from one
launch). Workload: 4096 rays x 400 zones, 21 bins, 32 x 64 quadrature, 3 species (seeded
synthetic rays). One entry = one Phi_l(eps_i, eps_j) of one zone and one l: Z N^2 2 per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--mode fwd+jac|fwd|spectral|solve]

`--mode solve` times the consumer of those Jacobians instead: the batched block-tridiagonal solve
of the per-ray Newton systems (sec. 2.1), 304 rays x 400 zones with m = 84 unknowns per zone (J and
H of nu_e and nu_ebar in 21 bins), FP32 block LU + two FP64 refinement sweeps per step.

Under torchrun every rank runs its own independent copy of the workload (weak scaling, no
collective on the data path); the time is the max over ranks. `--impl reference` times the FP64
CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import vx_inputs  # noqa: E402

WORKLOAD = 4
METRIC = "pair-kernel entries/s (zone*eps*eps'*l), FP32+adj vs FP64 fwd, % FP peak"
UNIT = "entries/s"


def entries(Z, N):
    return Z * N * N * 2


# DRAM bytes (read + write) per zone of the forward + tangent kernel, from one ncu capture of the
# 200-ray case of this workload (dram__bytes_read.sum + dram__bytes_write.sum = 91.0 + 591.6 MB
# for 80,000 zones, profiles/k_pair_mixed_tangents_200rays_pipes.md); scaled to a launch by the
# zone count. Set to None whenever the kernel changes, until it has been captured again.
TRAFFIC_BYTES_PER_ZONE = 8532
def measured_hbm_gbs():
    """The HBM copy bandwidth measured on this machine's GPUs (MEASURED_PEAKS.json), else the
    recipe's fallback figure; returns (GB/s, note)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs, a copy)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "of fallback (6.8 TB/s)"


# rays of the default workload in --mode spectral (410k zones: 17 GB of blocks)
SPECTRAL_RAYS = 1024


def algorithmic_flops_per_node(adj: bool) -> int:
    """Algorithmic FP32 operations per (zone, unordered bin pair, omega, E) node of the quadrature,
    counting an FMA as 2 and an exp, reciprocal, add or multiply as 1 (the count of the method,
    independent of how the kernel formulates it): the node's energy (1 FMA), the two Fermi-Dirac
    arguments (2 FMA), two exponentials and one reciprocal, the blocking product (2 FMA), the two
    quadratic kinematic factors (4 FMA) and the accumulation (2 FMA): 22 forward; the tangents
    add about 6 FMA per node (12), 34 in all. Only unordered bin pairs are integrated, since the
    exchange symmetry K_II(i, j) = K_I(j, i) is exact."""
    return 34 if adj else 22


def formulation_flops_per_node(adj: bool) -> int:
    """FP32 operations per node in the formulation the kernel evaluates (nodes in mirror pairs
    tau, -tau; tangents from r^2), same counting: forward 14; with tangents 38: the forward node
    plus E (2), r^2 and the four blocked products (6), the T and eta integrands (4) and their six
    moment FMAs (12); the production tangent's moments follow per (pair, omega) unit as
    q0 M(O) - M(GTa)."""
    return 38 if adj else 14


# Pipe utilisation of the benchmark's kernels from one ncu capture each (see profiles/; set to
# None whenever the kernel changes, until it has been captured again): the MUFU (XU) issue
# fraction of the forward + tangent kernel and the FP64-pipe fraction of the plain FP64 kernel.
MUFU_FRAC_TANGENT = 0.2530   # profiles/k_pair_mixed_tangents_200rays_pipes.md
FP64_FRAC_FP64FWD = 0.9154   # profiles/k_pair_mixed_tangents_and_k_pair_fp64_pipes_20rays.md
# fraction of the workload's zones the plain FP64 comparison leg evaluates, and its timed launches
FP64_SAMPLE_FRAC, FP64_REPEATS = 0.05, 3
# timed launches of the precise-mode leg (after two untimed ones)
PRECISE_REPEATS = 3


def rank_batch(rank: int, rays=None, workload: int = WORKLOAD) -> dict:
    """Each rank evaluates its own independent copy of the workload (seed = rank): weak scaling,
    no data exchanged between ranks."""
    return vx_inputs.make_batch(workload, seed=rank, rays=rays)


def max_over_ranks(ms_local: float, world: int, dist=None, device="cpu") -> float:
    """Step time of the whole job: the slowest rank's (all_reduce MAX; identity on one rank)."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(entries_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: all ranks' entries over the slowest rank's step time."""
    return entries_per_rank * world / (ms / 1000.0)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while active."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 7 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 7 and r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in self.rows if len(r) >= 7 for n, v in zip(names, r[3:7]) if v == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def oracle_sample_rate(b, n_zones: int, jac: bool, spectral: bool = False):
    """Entries/s of the FP64 oracle on the first n_zones zones of a batch (all host threads)."""
    import oracle
    oracle.build()
    sl = slice(0, n_zones)
    t0 = time.perf_counter()
    out = oracle.evaluate(b["eps"], b["n_mu"], b["n_e"], b["species"], b["state"][sl], b["J"][sl], b["H"][sl],
                          jac=jac, spectral=spectral)
    dt = time.perf_counter() - t0
    return entries(n_zones, len(b["eps"])) / dt, out["threads"], dt


def sized_sample(run, cap: int, n0: int, target_s: float):
    """Runs run(n) -> (rate, threads, seconds) on growing samples until one takes at least half of
    target_s (or the sample reaches cap); a small first sample overestimates the per-unit cost."""
    n = min(cap, n0)
    rate, thr, dt = run(n)
    while dt < 0.5 * target_s and n < cap:
        n = int(min(cap, max(n + 1, n * target_s / max(dt, 1e-3))))
        rate, thr, dt = run(n)
    return rate, thr, dt, n


def cpu_baseline(target_s: float = 15.0, workload: int = WORKLOAD, jac: bool = True, spectral: bool = False):
    b = vx_inputs.make_batch(workload, rays=range(16))
    rate, thr, dt, n = sized_sample(lambda k: oracle_sample_rate(b, k, jac, spectral), len(b["state"]), 64, target_s)
    what = "forward + Jacobian" if jac else ("forward + spectral blocks" if spectral else "forward")
    return {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": f"first {n} zones of workload {workload} (rays 0-15), {what}, FP64, {dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    b = vx_inputs.make_batch(WORKLOAD, rays=[0, 1])
    # per step: a bounded sample sized to a few seconds of all host cores
    _, thr, dt = oracle_sample_rate(b, 8, True)
    n = int(min(len(b["state"]), max(8, 8 * 4.0 / max(dt, 1e-3))))
    for _ in range(args.warmup):
        oracle_sample_rate(b, min(n, 8), True)
    t = []
    for _ in range(args.steps):
        r, thr, dt = oracle_sample_rate(b, n, True)
        t.append(dt)
    ms = 1000 * float(np.mean(t))
    value = entries(n, len(b["eps"])) / (ms / 1000)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": vx_inputs.WORKLOADS[WORKLOAD]["name"] + " forward+jacobian",
                       "zones_per_step": n, "bins": 21, "quadrature": "32x64", "species": 3},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": f"first {n} zones of workload {WORKLOAD} per step, forward + Jacobian"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


SOLVE_RAYS, SOLVE_ZONES, SOLVE_BINS, SOLVE_REFINE = 304, 400, 21, 2
SOLVE_METRIC = "Newton block rows solved/s (per-ray block-tridiagonal, FP32 LU + FP64 refinement)"


def solve_oracle_rate(s, rays):
    from oracle import btd as obtd
    o = s["offsets"]
    t0 = time.perf_counter()
    obtd.solve(s["A"], s["B"], s["C"], s["d"], o, rays=rays)
    dt = time.perf_counter() - t0
    return sum(int(o[r + 1] - o[r]) for r in rays) / dt, dt


def run_solve(args):
    import torch
    import torch.distributed as dist
    from vx_inputs import btd as gen

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    n_rays = args.rays or SOLVE_RAYS
    n_zones = args.zones or SOLVE_ZONES  # zones per ray
    if args.impl == "reference":
        if rank != 0:
            return 0
        s = gen.newton_system([n_zones] * 2, n_bins=SOLVE_BINS, seed=0)
        for _ in range(args.warmup):
            solve_oracle_rate(s, [0])
        t = [solve_oracle_rate(s, [0, 1])[1] for _ in range(args.steps)]
        ms = 1000 * float(np.mean(t))
        value = 2 * n_zones / (ms / 1000)
        print(json.dumps({"impl": "reference", "metric": SOLVE_METRIC, "value": value, "unit": "zones/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": f"2 rays x {n_zones} zones, m = 84"},
                          "cpu_baseline": {"value": value, "unit": "zones/s", "cores": 1, "kind": "oracle",
                                           "sample": "2 rays per step, banded LU (scipy solve_banded)"},
                          "e2e": {"value": value, "unit": "zones/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return 0
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    from paper_1404_1719_gb300 import BlockTridiagSolver, _build
    _build.build()
    s = gen.newton_system([n_zones] * n_rays, n_bins=SOLVE_BINS, seed=rank)
    m, Z = s["m"], s["d"].shape[0]
    host = {k: torch.from_numpy(np.ascontiguousarray(s[k])).pin_memory() for k in ("offsets", "A", "B", "C", "d")}
    dv = {k: v.to(dev) for k, v in host.items()}
    sv = BlockTridiagSolver(m, Z, SOLVE_REFINE)
    stream = torch.cuda.current_stream()
    x = torch.empty_like(dv["d"])

    def step():
        sv.solve(dv["offsets"], dv["A"], dv["B"], dv["C"], dv["d"], out=x)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert sv.check(), "numeric flag raised during warm-up"
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms_local = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms_local, world, dist, dev)
    ok = sv.check()
    # residual of the last solve, on the device in FP64 (a property that holds at any size)
    Ad, Bd, Cd, dd = dv["A"], dv["B"], dv["C"], dv["d"]
    r = dd - torch.einsum("zij,zj->zi", Bd, x)
    first = torch.zeros(Z, dtype=torch.bool, device=dev)
    first[dv["offsets"][:-1].long()] = True
    last = torch.roll(first, -1)
    r[1:] -= torch.where(first[1:, None], 0.0, torch.einsum("zij,zj->zi", Ad[1:], x[:-1]))
    r[:-1] -= torch.where(last[:-1, None], 0.0, torch.einsum("zij,zj->zi", Cd[:-1], x[1:]))
    rel_res = float(r.abs().max() / dd.abs().max())
    # end to end: pinned host blocks -> device -> solve -> host solution
    e2e_steps = max(1, min(3, args.steps))
    sv.solve_host(host["offsets"], host["A"], host["B"], host["C"], host["d"], device=dev)
    t_e2e = time.perf_counter()
    for _ in range(e2e_steps):
        sv.solve_host(host["offsets"], host["A"], host["B"], host["C"], host["d"], device=dev)
    ms_e2e = 1000.0 * (time.perf_counter() - t_e2e) / e2e_steps
    ms_e2e = max_over_ranks(ms_e2e, world, dist, dev)
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = x.numel() * x.element_size()
    if rank == 0:
        c = clk.summary()
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = c["sm_mhz"] or 2070.0
        peak = nsm * 128 * 2 * mhz * 1e6 / 1e12
        # FP32 flops of the block factorisation: Schur update A_k G_{k-1} (2 m^3) on every zone but a
        # ray's first, LU of D_k (2 m^3 / 3) on every zone, G_k = D_k^{-1} C_k (m elimination steps over
        # the m x m right-hand block, 2 m^3) on every zone but a ray's last; the O(m^2) sweeps and FP64
        # residuals are not counted
        flops = (Z - n_rays) * 2.0 * m ** 3 + Z * 2.0 * m ** 3 / 3.0 + (Z - n_rays) * 2.0 * m ** 3
        achieved = flops / (ms_local / 1000) / 1e12
        line = {
            "metric": SOLVE_METRIC, "value": job_rate(Z, world, ms), "unit": "zones/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{n_rays} rays x {n_zones} zones, block-tridiagonal Newton systems, "
                                   f"m = {m} (J, H of nu_e, nu_ebar x {SOLVE_BINS} bins)",
                       "zones": Z, "m": m, "n_refine": SOLVE_REFINE,
                       "l2": "inputs larger than L2 (A, B, C: %.1f GB)" % (3 * s["A"].nbytes / 1e9)},
            "e2e": {"value": job_rate(Z, world, ms_e2e), "unit": "zones/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "call": "BlockTridiagSolver.solve_host (pinned host tensors)",
                    "ms_per_step": ms_e2e},
            "gpu_launches": args.steps * (3 + 2 * SOLVE_REFINE),  # validate, factor, sweep; resid + sweep each
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None,
                         "note": "FP32 flops of the block factorisation over the whole step (factor kernel, "
                                 "sweeps and FP64 residuals); the factor kernel's pivot steps are sequential",
                         "peak_note": f"FP32 {nsm} SMs x 128 FMA x 2 x {mhz:.0f} MHz (median SM clock in the run)",
                         "kernel": "k_btd_factor + k_btd_sweep + k_btd_resid"},
            "residual_max_rel": rel_res,
            "clocks": c,
            "numeric_ok": bool(ok),
        }
        if not args.no_cpu:
            sub = gen.newton_system([n_zones] * n_rays, n_bins=SOLVE_BINS, seed=rank, rays=range(64))

            def run_rays(k):
                r, t = solve_oracle_rate(sub, list(range(k)))
                return r, 1, t

            rate, _, dt, k = sized_sample(run_rays, 64, 4, 12.0)
            line["cpu_baseline"] = {"value": rate, "unit": "zones/s", "cores": 1, "kind": "oracle",
                                    "sample": f"rays 0-{k - 1} of the workload, banded LU (scipy solve_banded), "
                                              f"{dt:.1f} s"}
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    sv.close()
    return 0


NES_METRIC = "NES kernel entries/s (zone*eps*eps'*l), FP32 forward+Jacobian, % FP peak"
# DRAM bytes (read + write) per zone of the NES forward + Jacobian kernel, from one ncu capture of
# the 256-ray case of the workload (108.8 + 765.1 MB for 102,400 zones,
# profiles/k_nes_tangents_20_and_64rays.md); None whenever the kernel changes, until captured again.
NES_TRAFFIC_BYTES_PER_ZONE = 8534
NES_N_MU, NES_N_E = 16, 48


def nes_oracle_rate(b, n_zones):
    import oracle
    oracle.build()
    sl = slice(0, n_zones)
    t0 = time.perf_counter()
    out = oracle.nes_evaluate(b["eps"], NES_N_MU, NES_N_E, b["species"], b["state"][sl], b["J"][sl], b["H"][sl],
                              jac=True)
    dt = time.perf_counter() - t0
    return entries(n_zones, len(b["eps"])) / dt, out["threads"], dt


def nes_placed_nodes(b, n_mu, n_e, stride=64):
    """Electron-energy nodes of a step that carry weight: the Laguerre panel always, the two
    Gauss-Legendre panels only where they are not empty (their upper ends above E_min), per
    (zone, bin pair in the down-scattering order, cos(omega) node); counted on every stride-th
    zone and scaled to all zones."""
    eps = b["eps"]
    N = len(eps)
    t, _ = np.polynomial.legendre.leggauss(n_mu)
    i, j = np.tril_indices(N)
    e, ep = eps[i][:, None], eps[j][:, None]
    y = 1.0 - t[None, :]
    q0 = e - ep
    Q = np.sqrt(q0 * q0 + 2 * e * ep * y)
    emin = (e * ep * y / (Q + q0)).ravel()                       # per (pair, omega)
    q0 = np.broadcast_to(q0, Q.shape).ravel()
    st = b["state"][::stride]
    mu = (st[:, 0] * st[:, 1])[:, None]
    n_p = n_e // 3
    p2 = (mu > emin[None, :]) & (q0[None, :] > 0)                 # panel 2: between distinct edges
    p1 = (mu - q0[None, :] > emin[None, :])                       # panel 1: E_min below the lower edge
    per_zone = n_p * (1 + p1 + p2).sum(axis=1)
    return int(round(per_zone.mean() * b["state"].shape[0]))


def run_nes(args):
    """Inelastic neutrino-electron scattering: forward rates + Jacobian of every zone of workload 4's
    4096 rays x 400 zones (21 bins), 16 cos(omega) nodes x 48 electron-energy nodes (three panels)."""
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        b = vx_inputs.make_batch(WORKLOAD, rays=[0])
        _, thr, dt = nes_oracle_rate(b, 4)
        n = int(min(len(b["state"]), max(4, 4 * 4.0 / max(dt, 1e-3))))
        t = [nes_oracle_rate(b, n)[2] for _ in range(args.steps)]
        ms = 1000 * float(np.mean(t))
        value = entries(n, len(b["eps"])) / (ms / 1000)
        print(json.dumps({"impl": "reference", "metric": NES_METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": vx_inputs.WORKLOADS[WORKLOAD]["name"] + " NES forward+jacobian",
                                     "zones_per_step": n, "quadrature": f"{NES_N_MU}x{NES_N_E}"},
                          "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                                           "sample": f"first {n} zones of workload {WORKLOAD} per step"},
                          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return 0
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    from paper_1404_1719_gb300 import NesRates, _build, capi
    _build.build()
    b = rank_batch(rank, rays=None if args.rays is None else range(args.rays))
    Z, N, S = b["state"].shape[0], len(b["eps"]), len(b["species"])
    host = {k: torch.from_numpy(np.ascontiguousarray(b[k])).pin_memory() for k in ("state", "J", "H")}
    d = {k: v.to(dev) for k, v in host.items()}
    nes = NesRates(b["eps"], NES_N_MU, NES_N_E, species=b["species"])
    stream = torch.cuda.current_stream()
    out = {k: torch.empty((Z, S, N), dtype=torch.float64, device=dev) for k in ("j0", "chi0", "j1", "chi1")}
    jac = torch.empty((Z, S, N, 4, 3), dtype=torch.float64, device=dev)
    bt = nes._batch(d["state"], d["J"], d["H"], b["ray_offsets"])
    fwd = capi.vx_out(*(out[k].data_ptr() for k in ("j0", "chi0", "j1", "chi1")), None)

    def step():
        capi.vx_nes_adjoint(nes.handle, bt, jac.data_ptr(), fwd, stream.cuda_stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert nes.check(), "numeric flag raised during warm-up"
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms_local = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms_local, world, dist, dev)
    ok = nes.check()
    # end to end through the public API: pinned host inputs in, rates and Jacobian back to pinned host
    h_out = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in out.items()}
    h_jac = torch.empty(jac.shape, dtype=jac.dtype, pin_memory=True)

    def step_e2e():  # vx_nes_adjoint_host: chunks copied in, evaluated and copied back, overlapped
        nes.adjoint_host(host["state"], host["J"], host["H"], forward=True, ray_offsets=b["ray_offsets"],
                         out=h_out, jac=h_jac)

    step_e2e()
    e2e_steps = max(1, min(3, args.steps))
    t_e2e = time.perf_counter()
    for _ in range(e2e_steps):
        step_e2e()
    ms_e2e = max_over_ranks(1000.0 * (time.perf_counter() - t_e2e) / e2e_steps, world, dist, dev)
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = sum(v.numel() * v.element_size() for v in h_out.values()) + h_jac.numel() * h_jac.element_size()
    if rank == 0:
        c = clk.summary()
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = c["sm_mhz"] or 2070.0
        peak = nsm * 128 * 2 * mhz * 1e6 / 1e12
        nodes = nes_placed_nodes(b, NES_N_MU, NES_N_E)
        achieved = nodes * algorithmic_flops_per_node(True) / (ms_local / 1000) / 1e12
        value = job_rate(entries(Z, N), world, ms)
        line = {
            "metric": NES_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": vx_inputs.WORKLOADS[WORKLOAD]["name"] + " NES forward+jacobian (mixed)"
                                   + ("" if args.rays is None else f" [first {args.rays} rays]"),
                       "zones": Z, "bins": N, "quadrature": f"{NES_N_MU}x{NES_N_E} (3 electron-energy panels)",
                       "species": S, "l2": "inputs larger than L2 (J, H: %.2f GB)" % (2 * b["J"].nbytes / 1e9)},
            "e2e": {"value": job_rate(entries(Z, N), world, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
                    "call": "vx_nes_adjoint_host (host buffers, pinned; chunks overlapped with the kernel)"},
            "gpu_launches": args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "flop_per_node": algorithmic_flops_per_node(True), "nodes_per_step": nodes,
                         "nodes_note": "electron-energy nodes the three-panel rule places (empty panels, where "
                                       "the Fermi edges lie below E_min, have none), counted on a 1-in-64 zone "
                                       "sample and scaled",
                         "traffic": NES_TRAFFIC_BYTES_PER_ZONE * Z if NES_TRAFFIC_BYTES_PER_ZONE else None,
                         "traffic_note": "ncu DRAM read+write of a 102,400-zone capture, scaled by zone count",
                         "peak_note": f"FP32 {nsm} SMs x 128 FMA x 2 x {mhz:.0f} MHz (median SM clock in the run)",
                         "kernel": f"k_nes<float, tangents, {NES_N_E // 3} nodes per panel>"},
            "clocks": c, "numeric_ok": bool(ok),
        }
        if not args.no_cpu:
            bb = vx_inputs.make_batch(WORKLOAD, rays=range(48))
            rate, thr, dt, n = sized_sample(lambda k: nes_oracle_rate(bb, k), len(bb["state"]), 256, 15.0)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
                                    "sample": f"first {n} zones of workload {WORKLOAD}, NES forward + Jacobian, "
                                              f"FP64, {dt:.1f} s"}
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    nes.close()
    return 0


ABS_METRIC = "absorption/emission rate entries/s (zone*species*eps), forward+Jacobian, % HBM peak"
# DRAM bytes (read + write) per entry (zone, species, bin) of the absorption rates + Jacobian kernel,
# from one ncu capture of the 1024-ray case of the workload (13.4 + 3241.5 MB for 25.8 M entries,
# profiles/k_abs_tangents_1024rays.md); None whenever the kernel changes, until captured again.
ABS_TRAFFIC_BYTES_PER_ENTRY = 126.1


def abs_oracle_rate(b, n_zones):
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.abs_evaluate(b["eps"], b["species"], b["state"][:n_zones], jac=True)
    dt = time.perf_counter() - t0
    return n_zones * len(b["species"]) * len(b["eps"]) / dt, 1, dt


def run_abs(args):
    """Charged-current absorption and emission on free nucleons: rates + Jacobian of every zone of
    workload 4's 4096 rays x 400 zones (21 bins, 3 species)."""
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        b = vx_inputs.make_batch(WORKLOAD, rays=range(64))
        for _ in range(args.warmup):
            abs_oracle_rate(b, 400)
        t = [abs_oracle_rate(b, len(b["state"]))[2] for _ in range(args.steps)]
        ms = 1000 * float(np.mean(t))
        n = len(b["state"])
        value = n * len(b["species"]) * len(b["eps"]) / (ms / 1000)
        print(json.dumps({"impl": "reference", "metric": ABS_METRIC, "value": value, "unit": "entries/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic",
                          "config": {"workload": vx_inputs.WORKLOADS[WORKLOAD]["name"] + " absorption+jacobian",
                                     "zones_per_step": n},
                          "cpu_baseline": {"value": value, "unit": "entries/s", "cores": 1, "kind": "oracle",
                                           "sample": f"first {n} zones of workload {WORKLOAD} per step"},
                          "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return 0
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    from paper_1404_1719_gb300 import AbsRates, _build, capi
    _build.build()
    b = rank_batch(rank, rays=None if args.rays is None else range(args.rays))
    Z, N, S = b["state"].shape[0], len(b["eps"]), len(b["species"])
    h_state = torch.from_numpy(np.ascontiguousarray(b["state"])).pin_memory()
    state = h_state.to(dev)
    ab = AbsRates(b["eps"], species=b["species"])
    stream = torch.cuda.current_stream()
    keys = ("j0", "chi0", "j1", "chi1")
    out = {k: torch.empty((Z, S, N), dtype=torch.float64, device=dev) for k in keys}
    jac = torch.empty((Z, S, N, 4, 3), dtype=torch.float64, device=dev)
    offs = torch.from_numpy(np.asarray(b["ray_offsets"], dtype=np.int32)).to(dev)
    bt = ab._state_batch(state, offs, None)
    fwd = capi.vx_out(*(out[k].data_ptr() for k in keys), None)

    def step():
        capi.vx_abs_adjoint(ab.handle, bt, jac.data_ptr(), fwd, stream.cuda_stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert ab.check(), "numeric flag raised during warm-up"
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms_local = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms_local, world, dist, dev)
    ok = ab.check()
    # end to end through the public API: the state in from pinned host memory, rates and Jacobian back
    h_out = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in out.items()}
    h_jac = torch.empty(jac.shape, dtype=jac.dtype, pin_memory=True)

    def step_e2e():
        state.copy_(h_state, non_blocking=True)
        res = ab.adjoint(state, forward=True, ray_offsets=offs)
        for k in keys:
            h_out[k].copy_(res[k], non_blocking=True)
        h_jac.copy_(res["jac"], non_blocking=True)
        torch.cuda.current_stream().synchronize()

    step_e2e()
    e2e_steps = max(1, min(3, args.steps))
    t_e2e = time.perf_counter()
    for _ in range(e2e_steps):
        step_e2e()
    ms_e2e = max_over_ranks(1000.0 * (time.perf_counter() - t_e2e) / e2e_steps, world, dist, dev)
    h2d = h_state.numel() * h_state.element_size()
    d2h = sum(v.numel() * v.element_size() for v in h_out.values()) + h_jac.numel() * h_jac.element_size()
    if rank == 0:
        c = clk.summary()
        ents = Z * S * N
        algo_bytes = Z * 32 + ents * 16 * 8  # the state read; four rates and twelve Jacobian entries written
        achieved = algo_bytes / (ms_local / 1000) / 1e9
        peak, peak_note = measured_hbm_gbs()
        line = {
            "metric": ABS_METRIC, "value": ents * world / (ms / 1000), "unit": "entries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 (FP32 occupation factors)", "data": "synthetic",
            "config": {"workload": vx_inputs.WORKLOADS[WORKLOAD]["name"] + " absorption/emission forward+jacobian"
                                   + ("" if args.rays is None else f" [first {args.rays} rays]"),
                       "zones": Z, "bins": N, "species": S,
                       "l2": "each step writes %.1f GB (> L2), which evicts the %.2f GB state between steps"
                             % (ents * 16 * 8 / 1e9, Z * 32 / 1e9)},
            "e2e": {"value": ents * world / (ms_e2e / 1000), "unit": "entries/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
                    "call": "AbsRates.adjoint with the state copied in from and the outputs back to pinned host "
                            "tensors every step"},
            "gpu_launches": args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "bytes_per_step": algo_bytes,
                         "traffic": ABS_TRAFFIC_BYTES_PER_ENTRY * ents if ABS_TRAFFIC_BYTES_PER_ENTRY else None,
                         "peak_note": peak_note,
                         "bound_note": "streaming kernel: FP32 occupations on FP32-pair exponent arguments, "
                                       "32 zones per warp, Jacobian rows staged per warp in shared memory "
                                       "and stored contiguously (profiles/k_abs_tangents_1024rays.md)",
                         "kernel": "k_abs<mixed, tangents>"},
            "clocks": c, "numeric_ok": bool(ok),
        }
        if not args.no_cpu:  # the oracle is fast here: the sample can grow to the whole workload
            rate, thr, dt, n = sized_sample(lambda k: abs_oracle_rate(b, k), len(b["state"]), 20000, 15.0)
            line["cpu_baseline"] = {"value": rate, "unit": "entries/s", "cores": thr, "kind": "oracle",
                                    "sample": f"first {n} zones of workload {WORKLOAD}, absorption + Jacobian, "
                                              f"FP64, {dt:.1f} s"}
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    ab.close()
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    from paper_1404_1719_gb300 import PairRates, _build
    _build.build()

    spec = args.mode == "spectral"
    if spec and args.rays is None:
        args.rays = SPECTRAL_RAYS  # the blocks are 42 KB per zone at 21 bins: bound the buffers
    b = rank_batch(rank, rays=None if args.rays is None else range(args.rays), workload=args.workload)
    fwd_only = args.mode != "fwd+jac"  # the forward kernel (with the spectral epilogue in "spectral")
    # the autotuner's choice is reported from its cache file
    tune_file = os.environ.get("VX_AUTOTUNE_CACHE") or os.path.join(
        os.environ.get("TMPDIR", "/tmp"), f"vx_bench_tune_{os.getpid()}.json")
    os.environ["VX_AUTOTUNE_CACHE"] = tune_file
    Z, N, S = b["state"].shape[0], len(b["eps"]), len(b["species"])
    host = {k: torch.from_numpy(np.ascontiguousarray(b[k])).pin_memory() for k in ("state", "J", "H")}
    d = {k: v.to(dev) for k, v in host.items()}
    split = args.quad == "split"
    rates = PairRates(b["eps"], b["n_mu"], b["n_e"], species=b["species"], graph=True, autotune=True, split=split)
    stream = torch.cuda.current_stream()
    out = {k: torch.empty((Z, S, N), dtype=torch.float64, device=dev) for k in ("j0", "chi0", "j1", "chi1")}
    jac = torch.empty((Z, S, N, 4, 3) if not fwd_only else (1,), dtype=torch.float64, device=dev)
    spec_out = {}
    if spec:
        spec_out = {"blocks": torch.empty((Z, S, 4, N, N), dtype=torch.float64, device=dev),
                    "grad_J": torch.empty((Z, S, N), dtype=torch.float64, device=dev),
                    "grad_H": torch.empty((Z, S, N), dtype=torch.float64, device=dev)}
        seeds = torch.ones((Z, S, N), dtype=torch.float64, device=dev)
    from paper_1404_1719_gb300 import capi
    bt = rates._batch(d["state"], d["J"], d["H"], b["ray_offsets"])
    fwd = capi.vx_out(*(out[k].data_ptr() for k in ("j0", "chi0", "j1", "chi1")), None)

    gout = capi.vx_out(*([seeds.data_ptr()] * 4), None) if spec else None

    def step():
        if spec:
            capi.vx_rates_spectral(rates.handle, bt, gout, spec_out["grad_J"].data_ptr(), spec_out["grad_H"].data_ptr(),
                                   spec_out["blocks"].data_ptr(), fwd, stream.cuda_stream)
        elif fwd_only:
            capi.vx_rates_eval(rates.handle, bt, fwd, stream.cuda_stream)
        else:
            capi.vx_rates_adjoint(rates.handle, bt, None, jac.data_ptr(), None, fwd, stream.cuda_stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert rates.check(), "numeric flag raised during warm-up"
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms_local = e0.elapsed_time(e1) / args.steps
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(ms_local, world, dist, dev)
    ok = rates.check()

    # ---- end-to-end: pinned host inputs -> device -> fused pass -> host rates (+ Jacobian).
    # Every mode goes through the library's host-buffer call, which stages chunks of zones through
    # device memory and overlaps their copies with the kernels.
    e2e_steps = max(1, min(3, args.steps))
    h_out = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in out.items()}
    h_jac = torch.empty(jac.shape, dtype=jac.dtype, pin_memory=True)
    h_spec = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in spec_out.items()}
    offs_host = np.ascontiguousarray(b["ray_offsets"], dtype=np.int32)  # the host calls take host offsets
    hb = capi.vx_batch(n_rays=bt.n_rays, n_zones=Z, ray_offsets=offs_host.ctypes.data_as(capi._ip),
                       state=host["state"].data_ptr(), J=host["J"].data_ptr(), H=host["H"].data_ptr())
    hfwd = capi.vx_out(*(h_out[k].data_ptr() for k in ("j0", "chi0", "j1", "chi1")), None)
    h_seeds = torch.ones((Z, S, N), dtype=torch.float64, pin_memory=True) if spec else None
    hseeds = capi.vx_out(*([h_seeds.data_ptr()] * 4), None) if spec else None

    def step_e2e():
        if spec:
            capi.vx_rates_spectral_host(rates.handle, hb, hseeds, h_spec["grad_J"].data_ptr(),
                                        h_spec["grad_H"].data_ptr(), h_spec["blocks"].data_ptr(), hfwd)
        elif fwd_only:
            capi.vx_rates_eval_host(rates.handle, hb, hfwd)
        else:
            capi.vx_rates_adjoint_host(rates.handle, hb, h_jac.data_ptr(), hfwd)

    step_e2e()  # first use allocates the staging slots
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_e2e = time.perf_counter()
    for _ in range(e2e_steps):
        step_e2e()
    torch.cuda.synchronize()
    ms_e2e = 1000.0 * (time.perf_counter() - t_e2e) / e2e_steps
    ms_e2e = max_over_ranks(ms_e2e, world, dist, dev)
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = sum(v.numel() * v.element_size() for v in out.values()) + (0 if fwd_only else jac.numel() * jac.element_size())
    d2h += sum(v.numel() * v.element_size() for v in spec_out.values())
    h2d += h_seeds.numel() * h_seeds.element_size() * 4 if spec else 0

    line = None
    if rank == 0:
        value = job_rate(entries(Z, N), world, ms)
        # roofline of the one kernel of the step (FP32 pipe peak from the unit counts and clock)
        c = clk.summary()
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = c["sm_mhz"] or 2070.0
        peak = nsm * 128 * 2 * mhz * 1e6 / 1e12
        npair = N * (N + 1) // 2
        nodes = Z * npair * b["n_mu"] * b["n_e"]
        achieved = nodes * algorithmic_flops_per_node(not fwd_only) / (ms_local / 1000) / 1e12
        achieved_form = nodes * formulation_flops_per_node(not fwd_only) / (ms_local / 1000) / 1e12
        # measured pipe rates of this GPU (per SM per clock), for the probe-based peaks
        pipes = capi.vx_probe_pipes(stream.cuda_stream)
        peak_probe = pipes["ffma2"] * 2 * nsm * mhz * 1e6 / 1e12
        # FP64 forward-only comparison on a sample of the same workload, timed over repeated launches
        sub = min(max(1, int(round(FP64_SAMPLE_FRAC * Z))), Z)
        r64 = PairRates(b["eps"], b["n_mu"], b["n_e"], species=b["species"], precision="fp64")
        o64 = {k: torch.empty((sub, S, N), dtype=torch.float64, device=dev) for k in out}
        args64 = (d["state"][:sub], d["J"][:sub], d["H"][:sub])
        r64.evaluate(*args64, out=o64)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(FP64_REPEATS):
            r64.evaluate(*args64, out=o64)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / FP64_REPEATS
        v64 = entries(sub, N) / (ms64 / 1000)
        nodes64 = sub * npair * b["n_mu"] * b["n_e"]
        peak64 = pipes["dfma"] * 2 * nsm * mhz * 1e6 / 1e12
        ach64 = nodes64 * algorithmic_flops_per_node(False) / (ms64 / 1000) / 1e12
        r64.close()
        # the same step in the precise mode (VX_PRECISE), a few timed launches: its cost
        precise = None
        if not spec and not split:
            rp = PairRates(b["eps"], b["n_mu"], b["n_e"], species=b["species"], graph=True, autotune=True,
                           precise=True)
            btp = rp._batch(d["state"], d["J"], d["H"], b["ray_offsets"])

            def step_p():
                if fwd_only:
                    capi.vx_rates_eval(rp.handle, btp, fwd, stream.cuda_stream)
                else:
                    capi.vx_rates_adjoint(rp.handle, btp, None, jac.data_ptr(), None, fwd, stream.cuda_stream)

            for _ in range(2):
                step_p()
            torch.cuda.synchronize()
            p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p0.record(stream)
            for _ in range(PRECISE_REPEATS):
                step_p()
            p1.record(stream)
            torch.cuda.synchronize()
            msp = p0.elapsed_time(p1) / PRECISE_REPEATS
            precise = {"value": entries(Z, N) / (msp / 1000), "unit": UNIT, "ms_per_step": msp,
                       "time_vs_default": msp / ms_local, "numeric_ok": bool(rp.check()),
                       "what": "VX_PRECISE: exact electron arguments in every zone, double-float l = 1 and "
                               "eta-tangent sums; |g - o|/|o| <= 1e-5 wherever the sum cancels < 100x "
                               "(tests/test_gpu_precision.py)"}
            rp.close()
        tune = {}
        try:
            with open(tune_file) as f:
                tune = {k.split("kind=")[1].split(",")[0].split("+")[0]: v for k, v in json.load(f).items()
                        if f"N={N},n_mu={b['n_mu']},n_e={b['n_e']}," in k and ("+split" in k) == split}
        except (OSError, ValueError, IndexError):
            pass
        kind = "forward" if fwd_only else "tangents"
        minb = tune.get(kind, {}).get("minb", 2)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": vx_inputs.WORKLOADS[args.workload]["name"]
                       + (" forward+spectral derivatives (mixed; blocks, J/H VJP, rates)" if spec else
                          " forward (mixed)" if fwd_only else " forward+jacobian (mixed)")
                       + (", split rule" if split else "")
                       + ("" if args.rays is None else f" [first {args.rays} rays]"),
                       "zones": Z, "rays": int(len(b["ray_offsets"]) - 1), "bins": N,
                       "quadrature": f"{b['n_mu']}x{b['n_e']}", "species": S,
                       "l2": "inputs larger than L2 (J, H: %.2f GB)" % (2 * b["J"].nbytes / 1e9),
                       "graph": True, "autotune": True},
            "e2e": {"value": job_rate(entries(Z, N), world, ms_e2e), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "call": ("vx_rates_spectral_host" if spec else
                             "vx_rates_eval_host" if fwd_only else "vx_rates_adjoint_host") + " (host buffers, pinned)",
                    "ms_per_step": ms_e2e},
            "gpu_launches": args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "frac_survey": achieved / peak,
                         "frac_formulation": achieved_form / peak,
                         "frac_of_probe_peak": achieved / peak_probe,
                         "flop_per_node": {"algorithmic": algorithmic_flops_per_node(not fwd_only),
                                           "formulation": formulation_flops_per_node(not fwd_only)},
                         "nodes_per_step": nodes,
                         "mufu_frac": MUFU_FRAC_TANGENT if (not fwd_only and not split) else None,
                         "mufu_note": "ncu sm__inst_executed_pipe_xu.avg.pct_of_peak_sustained_active of the "
                                      "forward + tangent kernel (profiles/)",
                         "traffic": (TRAFFIC_BYTES_PER_ZONE * Z if (TRAFFIC_BYTES_PER_ZONE and args.workload == WORKLOAD
                                                                    and not fwd_only and not split) else None),
                         "traffic_note": "ncu DRAM read+write of an 80,000-zone capture, scaled by zone count "
                                         "(profiles/k_pair_mixed_tangents_200rays_pipes.md)",
                         "peak_note": f"FP32 {nsm} SMs x 128 FMA x 2 x {mhz:.0f} MHz (median SM clock in the run); "
                                      f"probe: {pipes['ffma2']:.1f} FP32 lanes/clk/SM with packed FMAs = "
                                      f"{peak_probe:.1f} TFLOP/s at the same clock",
                         "kernel": f"k_pair_mixed<{b['n_e']}, {kind}, "
                                   f"{128 if minb == 2 else (80 if fwd_only else 96)}-register budget>"},
            "autotune": tune,
            **({"hbm": {"algorithmic_bytes_per_step": h2d + d2h,
                        "achieved_gbs": (h2d + d2h) / (ms_local / 1000) / 1e9,
                        "note": "inputs read + rates, blocks and J/H gradients written, per step"}} if spec else {}),
            "fp64_fwd": {"value": v64, "unit": UNIT, "ms_per_launch": ms64, "launches_timed": FP64_REPEATS,
                         "sample": f"first {sub} zones ({100 * sub / Z:.1f} % of the workload), plain FP64 forward only",
                         "ratio_mixed_fwd_adj_over_fp64_fwd": value / world / v64,
                         "roofline": {"bound": "alu", "achieved": ach64, "peak": peak64, "unit": "TFLOP/s",
                                      "frac": ach64 / peak64,
                                      "peak_note": f"FP64 {nsm} SMs x {pipes['dfma']:.2f} DFMA/clk (probe) x 2 x "
                                                   f"{mhz:.0f} MHz",
                                      "fp64_frac": FP64_FRAC_FP64FWD,
                                      "fp64_note": "ncu sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active "
                                                   "of k_pair_fp64 (profiles/)"}},
            "pipes": pipes,
            "precise_mode": precise,
            "clocks": c,
            "numeric_ok": bool(ok),
        }
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(workload=args.workload, jac=not fwd_only, spectral=spec)
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    rates.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU-baseline leg")
    ap.add_argument("--workload", type=int, default=WORKLOAD, choices=sorted(vx_inputs.WORKLOADS),
                    help="synthetic workload (default 4: 4096 rays x 400 zones)")
    ap.add_argument("--mode", choices=["fwd+jac", "fwd", "spectral", "solve", "nes", "abs"], default="fwd+jac",
                    help="step = forward + Jacobian pass (default), forward rates only, forward + the "
                         "derivatives with respect to the spectra (blocks and J/H VJP), the per-ray "
                         "block-tridiagonal Newton solve, the inelastic neutrino-electron scattering "
                         "kernel (forward + Jacobian), or the absorption and emission rates on nucleons "
                         "(forward + Jacobian)")
    ap.add_argument("--quad", choices=["standard", "split"], default="standard",
                    help="discrete rule in electron energy: standard, or split at the Fermi edge (VX_QUAD_SPLIT)")
    ap.add_argument("--rays", type=int, default=None,
                    help="use only the first R rays of the workload (small cases for profiling)")
    ap.add_argument("--zones", type=int, default=None,
                    help="--mode solve: zones per ray (default 400; small cases for profiling)")
    args = ap.parse_args()
    if args.mode == "solve":
        return run_solve(args)
    if args.mode == "nes":
        return run_nes(args)
    if args.mode == "abs":
        return run_abs(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
