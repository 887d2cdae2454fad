#!/usr/bin/env python
"""Benchmark of the MO vgl hot path on the organic-chain workload.

Workload: 150 nuclei (C:N:O:H 56:10:9:75 on a self-avoiding chain), 1650
Cartesian AOs up to f, 300 occupied MOs, 600 electrons x 256 walkers,
eps = 1e-10 radial cutoff; seeded synthetic inputs (no dataset exists here).
Metric: electron*MO vgl evaluations per second, N_elec * N_walk * N_mo / t,
one evaluation = value, gradient and Laplacian of one MO at one electron.

A step = new electron coordinates (device, bumps the time stamp) followed by
the MO vgl evaluation: the ao_vgl kernel and the contraction, every step.
Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "organic150: 150 nuclei, 1650 AO (s-f), 300 MO, 600 e- x 256 walkers, eps=1e-10"
METRIC = "electron·MO vgl evals/s (600 e-, 256 walkers) vs plain FP32 path; % roofline"
UNIT = "evals/s"
CPU_SAMPLE_POINTS = 2400     # 4 walkers: about 10 s of oracle work on one core


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["bf16x3", "tf32", "fp32", "fp64"], default="bf16x3")
    ap.add_argument("--no-fp32-line", action="store_true",
                    help="skip the plain FP32 path measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the uneven multi-molecule batch measurement")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the secondary measurements (large cluster, adjoint, cusp, "
                         "density, single moves)")
    ap.add_argument("--extra", default="large,adjoint,cusp,density,single_move",
                    help="comma-separated secondary measurements to run (profiling captures)")
    ap.add_argument("--walkers", type=int, default=None,
                    help="fewer walkers than the workload's 256 (profiling captures only)")
    return ap.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------- clocks ---
class ClockSampler:
    """nvidia-smi samples during the timed region (median SM clock, reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once the sampler is running
            t0 = time.monotonic()
            while not self.lines and self.proc.poll() is None and time.monotonic() - t0 < 5.0:
                time.sleep(0.01)
        except OSError:
            self.proc = None
        self.first = len(self.lines)
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        """Samples taken inside the timed region; when the region is shorter
        than the sampling interval, the last sample before it (said so)."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = self.lines[self.first:]
        lines = inside or self.lines[max(self.first - 1, 0):self.first]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
               "reasons": sorted(reasons), "samples": len(inside)}
        if not inside:
            out["note"] = "timed region shorter than the 100 ms sampling interval: sample taken just before it"
        return out


# ------------------------------------------------------------ roofline ---
def screen_work(mol, points, block=2048):
    """Algorithmic work of ao_vgl (Eqs. 1-4 under the Eq. 3 test), counted on
    the host for the roofline: the (point, shell) pairs with at least one
    primitive below the threshold, the primitives evaluated, and the
    Cartesian AOs of those pairs.  FP64, r^2 = dx dx + dy dy + dz dz."""
    import numpy as np
    T = (mol.bits - 1) * math.log(2.0) if mol.eps is None else -math.log(mol.eps)
    pts = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    nprim = np.asarray(mol.shell_prim_num, dtype=np.int64)
    prim_nuc = np.repeat(np.asarray(mol.shell_nucleus, dtype=np.int64), nprim)
    first = np.concatenate([[0], np.cumsum(nprim)[:-1]])
    lq = np.asarray(mol.shell_ang_mom, dtype=np.int64)
    ncart = (lq + 1) * (lq + 2) // 2
    gam = np.asarray(mol.exponent, dtype=np.float64)
    R = np.asarray(mol.nucl_coord, dtype=np.float64)
    pairs = prims = aos = 0
    for b in range(0, pts.shape[0], block):
        d = pts[b:b + block, None, :] - R[None, :, :]
        r2 = d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2]
        ev = (gam[None, :] * r2[:, prim_nuc]) < T
        per_shell = np.add.reduceat(ev.astype(np.int32), first, axis=1)
        live = per_shell > 0
        pairs += int(live.sum())
        prims += int(per_shell.sum())
        aos += int((live * ncart[None, :]).sum())
    return pairs, prims, aos


def alu_peaks(peaks):
    """FP32 FMA and MUFU (ex2) rates from unit counts and the maximum SM
    clock: 152 SMs x 128 FP32 lanes x 2 flop, and 16 MUFU results per SM per
    clock (4 per sub-partition)."""
    hz = peaks.get("sm_max_mhz", 2070.0) * 1e6
    return 152 * 128 * 2 * hz / 1e12, 152 * 16 * hz / 1e12


def roofline(mode, mol, ms_per_launch, peaks, stats=None, sparsity=None, work=None):
    """Roofline entries for the two kernels, from algorithmic work per launch.

    Dense modes: every (point, AO) entry.  Tensor-core modes skip blocks of
    screened AOs: ao_vgl's algorithmic bytes are those of the nonzero
    (point, AO) entries (the live 16-AO groups it actually writes are given
    beside them; stats = (live blocks, all blocks, live entries)).
    The contraction's algorithmic work is the sparse product of Sec. 3.2:
    2 * 5 * mo_num * nnz flops (one product; the bf16 split issues three,
    counted under issued_*) with nnz the nonzero
    (point, AO) pairs (sparsity = (live 16-AO groups, nnz)), over the bytes
    it must move (nonzero AO entries, C, the FP32 output).  Its bound is the
    roofline whose floor is longer (arithmetic intensity against the ridge
    point); both fractions are given.  The padded work the kernels actually
    move or issue is reported beside it.
    """
    P, na, nm = mol.point_num, mol.ao_num, mol.mo_num
    es = {"fp64": 8, "fp32": 4, "tf32": 4, "bf16x3": 4}[mode]
    nnz = P * na if sparsity is None else sparsity[1]
    ao_bytes = es * 5 * nnz
    dense = 2.0 * 5 * P * nm * na
    useful = 2.0 * 5 * nnz * nm
    out = {}
    t_ao = ms_per_launch[0] * 1e-3
    if t_ao > 0:
        a = ao_bytes / t_ao / 1e9
        out["ao_vgl"] = {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": a / peaks["hbm_gbs"],
                         "algorithmic_bytes": ao_bytes,
                         "dense_equivalent_bytes": es * 5 * P * na}
        if stats is not None and sparsity is not None:
            # whole live 16-AO groups of 128 rows, plus the mask bytes
            out["ao_vgl"]["written_bytes"] = sparsity[0] * 128 * 16 * es + stats[1]
            out["ao_vgl"]["live_block_fraction"] = stats[0] / stats[1]
        if work is not None and mode != "fp64":
            # per evaluated primitive one exp and ~5 FMA; per Cartesian AO of
            # a surviving pair ~14 flop (value, gradient, Laplacian assembly)
            fp32, mufu = alu_peaks(peaks)
            flops = 10.0 * work[1] + 14.0 * work[2]
            t_fma, t_xu = flops / (fp32 * 1e12), work[1] / (mufu * 1e12)
            t_alu = max(t_fma, t_xu)
            out["ao_vgl"]["alu"] = {
                "pairs": work[0], "prims_evaluated": work[1], "cartesian_aos": work[2],
                "fp32_flops": flops, "mufu_ops": work[1],
                "fp32": {"achieved": flops / t_ao / 1e12, "peak": fp32, "unit": "TFLOP/s",
                         "frac": t_fma / t_ao},
                "mufu": {"achieved": work[1] / t_ao / 1e12, "peak": mufu, "unit": "Tops/s",
                         "frac": t_xu / t_ao},
                "frac": t_alu / t_ao,
                "peak_note": "152 SMs x (128 FP32 FMA, 16 MUFU) per clock x max clock"}
            # the roofline that binds is the one whose floor is the longer
            if t_alu > ao_bytes / (peaks["hbm_gbs"] * 1e9):
                unit = "fp32" if t_fma >= t_xu else "mufu"
                e = out["ao_vgl"]["alu"][unit]
                out["ao_vgl"].update({"bound": "alu", "achieved": e["achieved"],
                                      "peak": e["peak"], "unit": e["unit"], "frac": e["frac"]})
    t_mo = ms_per_launch[1] * 1e-3
    if t_mo > 0:
        hbm = peaks["hbm_gbs"]
        if mode in ("bf16x3", "tf32"):
            tensor = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
            # the method's own count is one product; the bf16 split issues
            # three (hi*hi + hi*lo + lo*hi), reported under issued_* only
            fl = useful
            if mode == "bf16x3":
                tnote = "measured bf16 sustained"
            else:
                tensor = tensor * 0.5
                tnote = "measured bf16 sustained x 1/2 (tf32/bf16 nominal ratio)"
            # what the sparse product must move: the nonzero AO entries (both
            # bf16 planes, or FP32), C once, and the FP32 output
            nbytes = 4.0 * 5 * nnz + 4.0 * nm * na + 4.0 * 5 * P * nm
            t_hbm, t_tc = nbytes / (hbm * 1e9), fl / (tensor * 1e12)
            ent = {"algorithmic_flops": fl, "algorithmic_bytes": nbytes,
                   "arithmetic_intensity": fl / nbytes,
                   "ridge_flop_per_byte": tensor * 1e12 / (hbm * 1e9),
                   "dense_equivalent_flops": dense,
                   "split_products": 3 if mode == "bf16x3" else 1,
                   "tensor": {"achieved": fl / t_mo / 1e12, "peak": tensor, "unit": "TFLOP/s",
                              "frac": t_tc / t_mo, "peak_note": tnote},
                   "hbm": {"achieved": nbytes / t_mo / 1e9, "peak": hbm, "unit": "GB/s",
                           "frac": t_hbm / t_mo, "peak_note": "measured copy"}}
            # the roofline that binds is the one whose floor is the longer
            bound = "hbm" if t_hbm >= t_tc else "tensor"
            ent.update({"bound": bound, **{k: ent[bound][k] for k in
                                           ("achieved", "peak", "unit", "frac", "peak_note")}})
            if sparsity is not None:
                # one 128 x 16 x N_pad k-step per live (tile, 16-AO group);
                # N tiles of 160, the last one rounded up to 16
                nt = -(-nm // 160)
                n_pad = (nt - 1) * 160 + -(-(nm - (nt - 1) * 160) // 16) * 16
                issued = sparsity[0] * 128 * 16 * n_pad * 2.0 * (3 if mode == "bf16x3" else 1)
                ent["nnz_fraction"] = nnz / (P * na)
                ent["issued_flops"] = issued
                ent["issued_tflops"] = issued / t_mo / 1e12
                ent["issued_frac"] = issued / t_mo / 1e12 / tensor
            out["mo_contraction"] = ent
        else:
            if mode == "fp32":
                peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
                note = "152 SMs x 128 FP32 FMA/clk x max clock"
            else:
                peak, note = 1.25, "nominal GB300 FP64"
            a = useful / t_mo / 1e12
            out["mo_contraction"] = {"bound": "alu", "unit": "TFLOP/s", "peak": peak,
                                     "peak_note": note, "achieved": a, "frac": a / peak,
                                     "algorithmic_flops": useful,
                                     "dense_equivalent_flops": dense}
    return out


def speedup_decomposition(res, roof, mol):
    """The split-bf16 contraction's speedup over the plain FP32 SIMT GEMM,
    split into the work the block-sparse product skips and the rate at which
    the tensor cores do the rest (per product: the split issues three)."""
    mo = roof.get("mo_contraction", {})
    if "issued_flops" not in mo or not res.get("fp32_path"):
        return None
    dense = mo["dense_equivalent_flops"]
    per_product = mo["issued_flops"] / mo["split_products"]
    t32 = res["fp32_path"]["contraction_ms"] * 1e-3
    t16 = res["kernels"]["contraction_ms"] * 1e-3
    rate32 = dense / t32
    rate16 = per_product / t16
    return {"contraction_speedup": t32 / t16,
            "skipped_work_factor": dense / per_product,
            "rate_factor_per_product": rate16 / rate32,
            "fp32_simt_tflops": rate32 / 1e12,
            "split_bf16_tflops_per_product": rate16 / 1e12,
            "ao_vgl_speedup": (res["fp32_path"]["ao_vgl_ms"] / res["kernels"]["ao_vgl_ms"]
                               if res["kernels"]["ao_vgl_ms"] else None),
            "note": "contraction_speedup = skipped_work_factor x rate_factor_per_product"}


def traffic_for(kernel, mode):
    """DRAM bytes per launch from the committed ncu summary, if every source
    file of the kernel still hashes to what was captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        with open(path) as f:
            tab = json.load(f)
        ent = tab.get(f"{kernel}:{mode}")
        if not ent:
            return None
        import hashlib
        srcs = ent["source"] if isinstance(ent["source"], list) else [ent["source"]]
        hsh = hashlib.sha256()
        for src in srcs:
            with open(os.path.join(ROOT, src), "rb") as f:
                hsh.update(f.read())
        return ent["bytes_per_launch"] if hsh.hexdigest()[:16] == ent["source_sha"] else None
    except Exception:
        return None


# ----------------------------------------------------------- our arm ---
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2512_16677_gb300 import qmckl, synth

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
    mol = synth.make_config(2, walk_num=args.walkers)
    peaks, peak_src = load_peaks()
    coords = torch.from_numpy(mol.coord).cuda()
    g = torch.Generator(device="cpu").manual_seed(1234 + rank)
    step_disp = torch.randn(coords.shape, generator=g, dtype=torch.float64).cuda() * 0.05
    coord_set = [coords, coords + step_disp]        # two electron configurations

    def measure(mode, steps, warmup, timing=True):
        ctx = qmckl.Context(mode)
        ctx.set_molecule(mol)
        ctx.set_points_device(coord_set[0])
        out = ctx.mo_vgl_device()
        for i in range(warmup):
            ctx.set_points_device(coord_set[i % 2])
            ctx.mo_vgl_device(out)
        torch.cuda.synchronize()
        ctx.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        # the step is timed without the library's per-kernel events (they
        # cost about 2% of the step); the kernel times come from a second
        # pass of the same steps with the events on
        ctx.set_timing(False)
        ctx.kernel_count()
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clk:
            e0.record(stream)
            for i in range(steps):
                ctx.set_points_device(coord_set[i % 2])
                ctx.mo_vgl_device(out)
            e1.record(stream)
            torch.cuda.synchronize()
        ctx.synchronize()
        launches = ctx.kernel_count()
        if dist:
            dist.barrier()
        ms = e0.elapsed_time(e1)
        if dist:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        kms, kn = [0.0] * 3, [0] * 3
        if timing:
            ctx.set_timing(True)
            for i in range(steps):
                ctx.set_points_device(coord_set[i % 2])
                ctx.mo_vgl_device(out)
            torch.cuda.synchronize()
            ctx.synchronize()
            kms, kn = ctx.get_timing()
            ctx.set_timing(False)
        return ctx, out, ms, kms, kn, clk.summary(), launches

    evals_per_step = mol.elec_num * mol.walk_num * mol.mo_num
    ctx, out, ms, kms, kn, clocks, launches = measure(args.mode, args.steps, args.warmup)
    ms_step = ms / args.steps
    value = world * evals_per_step / (ms_step * 1e-3)
    per_launch = [kms[i] / kn[i] if kn[i] else 0.0 for i in range(3)]
    stats = ctx.block_stats() if args.mode in ("bf16x3", "tf32") else None
    sparsity = ctx.sparsity_stats() if args.mode in ("bf16x3", "tf32") else None
    # the library's last evaluation was of this point set
    work = screen_work(mol, coord_set[(args.steps - 1) % 2].cpu().numpy())
    roof = roofline(args.mode, mol, per_launch, peaks, stats, sparsity, work)
    dominant = max(roof, key=lambda k: per_launch[0 if k == "ao_vgl" else 1])
    dom = dict(roof[dominant])
    dom["kernel"] = dominant
    dom["traffic"] = traffic_for(dominant, args.mode)
    dom["peak_source"] = peak_src
    dom["ms_per_launch"] = per_launch[0 if dominant == "ao_vgl" else 1]

    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16x3": "bf16x3 (f32 accum)", "tf32": "tf32 (f32 accum)", "fp32": "f32",
                  "fp64": "f64"}[args.mode],
        "data": "synthetic (seeded organic-chain molecule, random MO coefficients)",
        "config": {"workload": WORKLOAD if args.walkers is None else
                   WORKLOAD.replace("x 256 walkers", f"x {mol.walk_num} walkers"),
                   "mode": args.mode, "points": mol.point_num,
                   "ao_num": mol.ao_num, "mo_num": mol.mo_num,
                   "l2": "inputs larger than L2 (AO tensor %.2f GB per step)" % (
                       5 * mol.point_num * mol.ao_num * 4 / 1e9),
                   "parallelism": f"walker replicas x{world}" if world > 1 else "1 GPU"},
        "roofline": dom,
        "kernels": {"ao_vgl_ms": per_launch[0], "contraction_ms": per_launch[1],
                    "points_ms": per_launch[2], "all": roof},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }

    # the main mode's first rows, kept for the accuracy comparison below
    samples = {}
    if rank == 0 and not args.no_cpu_baseline:
        # the timed steps alternate two configurations: evaluate the first one
        # (the oracle's sample) again
        ctx.set_points_device(coord_set[0])
        ctx.mo_vgl_device(out)
        samples[args.mode] = out.reshape(-1)[:CPU_SAMPLE_POINTS * 5 * mol.mo_num].double().cpu().numpy()

    # same workload through the other compute paths: the plain FP32 path
    # (SIMT ao_vgl + SIMT GEMM), TF32 tensor cores and FP64 (a few steps)
    if not args.no_fp32_line:
        del ctx
        ctx = None
        for mode, steps in (("fp32", max(3, args.steps // 4)), ("tf32", max(3, args.steps // 4)),
                            ("fp64", 3)):
            if mode == args.mode:
                continue
            co, oo, mso, ko, no, clko, _ = measure(mode, steps, 2)
            if rank == 0 and not args.no_cpu_baseline:
                co.set_points_device(coord_set[0])
                co.mo_vgl_device(oo)
            ms_o = mso / steps
            ent = {"value": world * evals_per_step / (ms_o * 1e-3), "ms_per_step": ms_o,
                   "steps": steps, "contraction_ms": ko[1] / max(no[1], 1),
                   "ao_vgl_ms": ko[0] / max(no[0], 1), "clocks": clko}
            if mode in ("bf16x3", "tf32", "fp64"):
                # block-sparse paths: the contraction against its roofline, from
                # the method's sparse count
                lt = [ko[i] / no[i] if no[i] else 0.0 for i in range(3)]
                r = roofline(mode, mol, lt, peaks, co.block_stats(), co.sparsity_stats(), None)
                ent["roofline"] = {k: r["mo_contraction"][k] for k in
                                   ("bound", "achieved", "peak", "unit", "frac")
                                   if k in r["mo_contraction"]}
            res[f"{mode}_path"] = ent
            if rank == 0 and not args.no_cpu_baseline:
                samples[mode] = oo.reshape(-1)[:CPU_SAMPLE_POINTS * 5 * mol.mo_num].double().cpu().numpy()
            del co, oo
        res["speedup_vs_fp32_path"] = res["fp32_path"]["ms_per_step"] / ms_step
        if args.mode == "bf16x3":
            res["speedup_decomposition"] = speedup_decomposition(res, roof, mol)
    res["_accuracy_samples"] = samples

    if not args.no_batch:
        res["batch"] = measure_batch(args, world)
    if not args.no_extra:
        extras = {"large": lambda: measure_large(args, world), "adjoint": lambda: measure_adjoint(args),
                  "cusp": lambda: measure_cusp(args), "density": lambda: measure_density(args),
                  "single_move": lambda: measure_single(args)}
        for name in [e for e in args.extra.split(",") if e]:
            if name not in extras:
                raise SystemExit(f"unknown --extra measurement {name!r}")
            res[name] = extras[name]()

    # end to end through the host-memory C-ABI calls: H2D of the coordinates
    # and D2H of the whole MO vgl tensor inside the timed region
    host_in = torch.empty(coords.shape, dtype=torch.float64, pin_memory=True)
    host_in.copy_(coords.cpu())
    host_out = torch.empty((mol.point_num * 5 * mol.mo_num,),
                           dtype=torch.float64 if args.mode == "fp64" else torch.float32,
                           pin_memory=True)
    ce = qmckl.Context(args.mode)
    ce.set_molecule(mol)
    hin, hout = host_in.numpy(), host_out.numpy()
    for _ in range(2):
        ce.set_points(hin)
        ce.mo_vgl(hout)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ce.set_points(hin)
        ce.mo_vgl(hout)
    torch.cuda.synchronize()
    te = (time.perf_counter() - t0) / args.e2e_steps
    if dist:
        t = torch.tensor([te], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        te = float(t.item())
    res["e2e"] = {"value": world * evals_per_step / te, "unit": UNIT,
                  "ms_per_step": te * 1e3,
                  "h2d_bytes_per_step": int(host_in.numel() * 8),
                  "d2h_bytes_per_step": int(host_out.numel() * host_out.element_size())}
    gpu_out_w0 = None
    if rank == 0 and not args.no_cpu_baseline:
        gpu_out_w0 = hout.reshape(-1, 5, mol.mo_num)[:CPU_SAMPLE_POINTS].astype(np.float64)
    ce.close()
    return res, mol, gpu_out_w0


def _batch_launches(n_mols):
    """Kernels of one batch step: a coordinate conversion per molecule, the
    point sort (cell keys, three kernels per 8-bit radix pass over the
    15-bit cell key below the molecule index, the gather), the reach
    pre-pass, ao_vgl and the contraction."""
    passes = -(-(15 + max(0, (n_mols - 1).bit_length())) // 8)
    return n_mols + (1 + 3 * passes + 1) + 3


def measure_batch(args, world):
    """Uneven batch: 12 chains of 20-200 nuclei, 4 e-/nucleus, 16-256 walkers,
    split-bf16; new points for every molecule + one batch run per step (the
    point sort, reach pre-pass, ao_vgl and contraction replayed from a CUDA
    graph)."""
    import torch
    from paper_2512_16677_gb300 import qmckl, synth
    mols = synth.make_config(4)
    coords = [torch.from_numpy(m.coord).cuda() for m in mols]
    moved = [c + 0.05 for c in coords]
    ctxs = []
    nnz = []
    for m, c in zip(mols, coords):
        ctx = qmckl.Context("bf16x3")
        ctx.set_molecule(m)
        ctx.set_points_device(c)
        ctx.mo_vgl_device()            # once on its own: the molecule's exact sparsity
        torch.cuda.synchronize()
        nnz.append(ctx.sparsity_stats()[1])
        ctxs.append(ctx)
    b = qmckl.Batch(ctxs)
    bn, tune_ms = b.autotune(reps=3)
    b.run()
    b.synchronize()
    evals = sum(m.elec_num * m.walk_num * m.mo_num for m in mols)
    steps = max(5, args.steps)
    for i in range(3):
        for c, x in zip(ctxs, coords if i % 2 else moved):
            c.set_points_device(x)
        b.run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    for i in range(steps):
        for c, x in zip(ctxs, coords if i % 2 else moved):
            c.set_points_device(x)
        b.run()
    e1.record(stream)
    torch.cuda.synchronize()
    b.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"workload": "12 chains, 20-200 nuclei, 220-2200 AOs, 4 e-/nucleus, 16-256 walkers, "
                        "eps=1e-10, bf16x3",
            "evals_per_step": evals, "points": sum(m.point_num for m in mols),
            "ms_per_step": ms, "value": world * evals / (ms * 1e-3), "unit": UNIT,
            "autotuned_bn_max": bn, "autotune_contraction_ms": tune_ms, "cuda_graph": True,
            "launches_per_step": _batch_launches(len(mols)),
            "roofline": batch_roofline(mols, nnz, tune_ms, load_peaks()[0])}


def batch_roofline(mols, nnz, ms, peaks):
    """The batch contraction (one launch over every molecule) against the
    roofline of its algorithmic work: per molecule the sparse count
    2 * 5 * N_mo * sum_p nnz_AO(p) (one product), over the bytes it must
    move (nonzero AO entries in two bf16 planes, C once, the FP32 output).
    nnz per molecule comes from the molecule's own evaluation."""
    fl = sum(2.0 * 5 * m.mo_num * z for m, z in zip(mols, nnz))
    nbytes = sum(4.0 * 5 * z + 4.0 * m.mo_num * m.ao_num + 4.0 * 5 * m.point_num * m.mo_num
                 for m, z in zip(mols, nnz))
    t = ms * 1e-3
    hbm = peaks["hbm_gbs"]
    tensor = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    t_hbm, t_tc = nbytes / (hbm * 1e9), fl / (tensor * 1e12)
    bound = "hbm" if t_hbm >= t_tc else "tensor"
    ent = {"kernel": "batch contraction", "algorithmic_flops": fl, "algorithmic_bytes": nbytes,
           "hbm": {"achieved": nbytes / t / 1e9, "peak": hbm, "unit": "GB/s", "frac": t_hbm / t},
           "tensor": {"achieved": fl / t / 1e12, "peak": tensor, "unit": "TFLOP/s",
                      "frac": t_tc / t},
           "bound": bound, "ms_per_launch": ms}
    ent.update({k: ent[bound][k] for k in ("achieved", "peak", "unit", "frac")})
    return ent


def _time_steps(fn, steps, warmup=2):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    s = torch.cuda.current_stream()
    e0.record(s)
    for _ in range(steps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def measure_large(args, world):
    """1000-nucleus cluster, 10 000 AOs, 2000 MOs, 4000 e- x 16 walkers:
    split-bf16 (block-sparse) against the plain FP32 path (dense)."""
    import torch
    from paper_2512_16677_gb300 import qmckl, synth
    mol = synth.make_config(5)
    coords = [torch.from_numpy(mol.coord).cuda()]
    coords.append(coords[0] + 0.05)
    evals = mol.elec_num * mol.walk_num * mol.mo_num
    out = {"workload": "cluster1000: 1000 nuclei, 10000 AO, 2000 MO, 4000 e- x 16 walkers, "
                       "eps=1e-10", "evals_per_step": evals}
    for mode, steps in (("bf16x3", max(3, args.steps // 2)), ("fp32", 2)):
        ctx = qmckl.Context(mode)
        ctx.set_molecule(mol)
        ctx.set_points_device(coords[0])
        o = ctx.mo_vgl_device()
        k = [0]

        def step():
            k[0] += 1
            ctx.set_points_device(coords[k[0] % 2])
            ctx.mo_vgl_device(o)
        ms = _time_steps(step, steps, warmup=1)
        ent = {"ms_per_step": ms, "value": world * evals / (ms * 1e-3)}
        if mode == "bf16x3":
            live, total, entries = ctx.block_stats()
            ent["live_block_fraction"] = live / total
            ent["live_entry_fraction"] = entries / (mol.point_num * mol.ao_num)
        out[mode] = ent
        del ctx, o
        torch.cuda.empty_cache()
    out["speedup_vs_fp32_path"] = out["fp32"]["ms_per_step"] / out["bf16x3"]["ms_per_step"]
    return out


def measure_adjoint(args):
    """C/H chain, 50 nuclei, 500 AOs, 100 MOs, 200 e- x 128 walkers: forward
    plus backward (dL/dC and dL/dR_nuc) per step, and the backward alone, in
    FP64, FP32 (SIMT products) and split bf16 (tensor-core products)."""
    import torch
    from paper_2512_16677_gb300 import qmckl, synth
    mol = synth.make_config(3)
    peaks, _ = load_peaks()
    coord = torch.from_numpy(mol.coord).cuda()
    res = {"workload": "chain50: 50 nuclei, 500 AO, 100 MO, 200 e- x 128 walkers"}
    rows = 5 * mol.point_num
    # the two products of the backward, one product each (the method's count)
    flops = 2.0 * 2 * rows * mol.mo_num * mol.ao_num
    for mode, steps in (("fp64", 3), ("fp32", 10), ("bf16x3", 10)):
        ctx = qmckl.Context(mode)
        ctx.set_molecule(mol)
        ctx.set_points_device(coord)
        o = ctx.mo_vgl_device()
        W = torch.randn(o.shape, dtype=o.dtype, device="cuda")

        def fwd_bwd():
            ctx.set_points_device(coord)
            ctx.mo_vgl_device(o)
            ctx.backward_device(W)

        def bwd():
            ctx.backward_device(W)
        ms = _time_steps(fwd_bwd, steps, warmup=1)
        mb = _time_steps(bwd, steps, warmup=1)
        ent = {"ms_per_fwd_bwd": ms, "ms_backward": mb,
               "evals_per_s": mol.elec_num * mol.walk_num * mol.mo_num / (ms * 1e-3),
               "products_flops": flops, "products_tflops": flops / (mb * 1e-3) / 1e12}
        if mode == "bf16x3":
            tensor = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
            # what the block-sparse backward must move at least: W in (FP32),
            # the forward's live AO blocks in (bf16 hi + lo, 32 KB each),
            # Abar at the live blocks out and back (FP32, 32 KB each), dL/dC
            live, total, _ = ctx.block_stats()
            blk = 128 * 64 * 4.0
            nbytes = 4.0 * rows * mol.mo_num + live * blk + 2 * live * blk + \
                8.0 * mol.mo_num * mol.ao_num
            ent["live_blocks"] = live
            ent["total_blocks"] = total
            ent["roofline"] = {
                "bound": "hbm", "achieved": nbytes / (mb * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": nbytes / (mb * 1e-3) / 1e9 / peaks["hbm_gbs"],
                "algorithmic_bytes": nbytes,
                "tensor": {"achieved": flops / (mb * 1e-3) / 1e12, "peak": tensor,
                           "unit": "TFLOP/s", "frac": flops / (mb * 1e-3) / 1e12 / tensor},
                "note": "whole backward (W gather and split, dL/dC and Abar products over the "
                        "live blocks, dR kernel) against the bytes W, the live AO blocks and "
                        "the live Abar blocks must move"}
        res[mode] = ent
        ctx.close()
    return res


def measure_cusp(args):
    """Organic chain step (bf16x3, 600 e- x 256 walkers) with the MO cusp
    correction of Sec. 3.3 at radii 0.5/sqrt(Z) bohr, against the same step
    without it; FP64 set-up of the coefficients timed once."""
    import numpy as np
    import torch
    from paper_2512_16677_gb300 import qmckl, synth
    mol = synth.make_config(2)
    rc = synth.cusp_radii(mol)
    coord = torch.from_numpy(mol.coord).cuda()
    pts = mol.points
    inside = 0
    for A in range(mol.nucl_num):
        d2 = ((pts - mol.nucl_coord[A]) ** 2).sum(1)
        inside += int((d2 < rc[A] ** 2).sum())
    res = {"workload": "organic150 step with the Sec. 3.3 cusp correction, radii 0.5/sqrt(Z) bohr",
           "point_sphere_pairs": inside}
    for on in (False, True):
        ctx = qmckl.Context("bf16x3")
        ctx.set_molecule(mol)
        ctx.set_points_device(coord)
        if on:
            ctx.set_mo_cusp(rc)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.cusp_coefficients_device()   # FP64 set-up of the coefficients
            torch.cuda.synchronize()
            res["setup_ms"] = (time.perf_counter() - t0) * 1e3
        o = ctx.mo_vgl_device()

        def step():
            ctx.set_points_device(coord)
            ctx.mo_vgl_device(o)
        res["ms_per_step_with" if on else "ms_per_step_without"] = _time_steps(step, 10, warmup=2)
    res["overhead_ms"] = res["ms_per_step_with"] - res["ms_per_step_without"]
    return res


def measure_single(args):
    """Single-electron moves on the organic chain (256 walkers): per move,
    the proposed positions of one electron in every walker go in and the MO
    vgl [256][5][300] at them comes out (device memory, one stream)."""
    import torch
    from paper_2512_16677_gb300 import qmckl, synth
    mol = synth.make_config(2)
    coord = torch.from_numpy(mol.coord).cuda()
    g = torch.Generator(device="cpu").manual_seed(99)
    moves = [(e, (coord[:, e, :] + 0.3 * torch.randn((mol.walk_num, 3), generator=g,
                                                      dtype=torch.float64).cuda()).contiguous())
             for e in range(0, mol.elec_num, 37)]
    res = {"workload": "organic150, 256 walkers, one electron moved per call, 300 MOs",
           "walkers": mol.walk_num}
    for mode in ("bf16x3", "fp64"):
        ctx = qmckl.Context(mode)
        ctx.set_molecule(mol)
        ctx.set_points_device(coord)
        ctx.mo_vgl_device()
        out = None
        k = [0]

        def move():
            nonlocal out
            e, p = moves[k[0] % len(moves)]
            k[0] += 1
            ctx.set_single_point_device(e, p)
            out = ctx.mo_vgl_single_device(out)
        ms = _time_steps(move, 200 if mode == "bf16x3" else 20, warmup=3)
        res[mode] = {"us_per_move": ms * 1e3,
                     "evals_per_s": mol.walk_num * mol.mo_num / (ms * 1e-3)}
        del ctx
    return res


def measure_density(args):
    """Density on a 100^3 grid (Sec. 5.4) for the 104-nucleus stand-in with
    1090 AOs and 218 doubly occupied MOs: one density evaluation per step,
    the grid built on the device."""
    import torch
    from paper_2512_16677_gb300 import qmckl, synth
    mol = synth.make_config(6)
    o, h, n = synth.density_grid(mol, n=100)
    ax = [torch.arange(n[k], dtype=torch.float64, device="cuda") * float(h[k]) + float(o[k])
          for k in range(3)]
    gx, gy, gz = torch.meshgrid(*ax, indexing="ij")
    grid = torch.stack([gx, gy, gz], -1).reshape(-1, 3).contiguous()
    w = synth.occupations(mol)
    res = {"workload": "100^3 grid, 104 nuclei, 1090 AOs, 218 doubly occupied MOs, eps=1e-10",
           "points": int(grid.shape[0])}
    for mode, steps in (("bf16x3", 10), ("tf32", 10), ("fp32", 3), ("fp64", 1)):
        ctx = qmckl.Context(mode)
        ctx.set_molecule(mol)
        ctx.set_points_device(grid)
        rho = ctx.density_device(w)
        ctx.set_timing(True)

        def step():
            ctx.density_device(w, rho)
        ms = _time_steps(step, steps, warmup=1)
        kms, kn = ctx.get_timing()
        res[mode] = {"ms_per_grid": ms, "points_per_s": grid.shape[0] / (ms * 1e-3),
                     "ao_values_ms": kms[0] / max(kn[0], 1), "contraction_ms": kms[1] / max(kn[1], 1)}
        del ctx
    return res


# -------------------------------------------------------- cpu baseline ---
_ORACLE_MEMO = {}


def oracle_sample(mol, n_points, memo=False):
    """Time the FP64 oracle on the first n_points of walker 0 (one thread);
    memo=True returns an earlier result for the same molecule and size."""
    key = (id(mol), n_points)
    if memo and key in _ORACLE_MEMO:
        return _ORACLE_MEMO[key]
    from oracle import oracle
    oracle.build()
    pts = mol.points[:n_points]
    t0 = time.perf_counter()
    ref, size = oracle.mo_vgl(mol, points=pts)
    dt = time.perf_counter() - t0
    _ORACLE_MEMO[key] = (ref, size, dt)
    return ref, size, dt


def host_cores():
    """Threads to run the oracle on: the cores this process may use."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_model():
    """The host CPU's model string (lscpu), e.g. for placing the baseline."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_parallel(mol, pts, threads):
    """Time the unchanged FP64 oracle over `threads` disjoint ranges of pts,
    one thread each (the oracle is C called through ctypes, which releases
    the GIL, so the threads run on separate cores)."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np
    from oracle import oracle
    oracle.build()
    parts = [p for p in np.array_split(pts, threads) if p.shape[0]]
    with ThreadPoolExecutor(max_workers=len(parts)) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda p: oracle.mo_vgl(mol, points=p), parts))
        dt = time.perf_counter() - t0
    return dt, len(parts)


def cpu_baseline(mol, gpu_w0):
    """The FP64 oracle on the host cores: all of them (the line's value) and
    one (single_core), on bounded samples of the workload's points."""
    n = CPU_SAMPLE_POINTS
    ref, size, dt = oracle_sample(mol, n)
    cores = host_cores()
    npar = min(mol.point_num, cores * (n // 4))
    dtp, used = oracle_parallel(mol, mol.points[:npar], cores)
    model = cpu_model()
    out = {"value": npar * mol.mo_num / dtp, "unit": UNIT, "cores": used,
           "kind": "oracle", "cpu_model": model,
           "sample": f"points 0-{npar - 1} of the 256-walker workload split over {used} "
                     f"threads ({n // 4} points each), screened FP64 oracle with compensated "
                     f"sums, {dtp:.1f} s wall",
           "single_core": {"value": n * mol.mo_num / dt, "unit": UNIT, "cores": 1,
                           "sample": f"walkers 0-{n // mol.elec_num - 1} ({n} points), "
                                     f"{dt:.1f} s"}}
    if gpu_w0 is not None:
        import numpy as np
        e = np.abs(gpu_w0.reshape(ref.shape) - ref) / (size + 1e-300)
        out["max_err_vs_oracle"] = {"value": float(e[:, 0].max()),
                                    "gradient": float(e[:, 1:4].max()),
                                    "laplacian": float(e[:, 4].max()),
                                    "metric": "normwise |gpu-oracle|/sum|C||chi|, "
                                              "same sample"}
    return out


def accuracy(mol, samples, main_mode):
    """Max normwise error against the FP64 oracle per compute path, on the
    first rows of each path's output (the CPU baseline's sample)."""
    import numpy as np
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from tolerances import TOL
    if not samples:
        return None
    n = CPU_SAMPLE_POINTS
    ref, size, _ = oracle_sample(mol, n, memo=True)
    out = {}
    for mode, got in samples.items():
        e = np.abs(got.reshape(ref.shape) - ref) / (size + 1e-300)
        out[mode] = {"value": float(e[:, 0].max()), "gradient": float(e[:, 1:4].max()),
                     "laplacian": float(e[:, 4].max()), "stated_bar": TOL[mode][0]}
    out["metric"] = "normwise |gpu-oracle|/sum|C||chi| on the first %d points" % n
    return out


def common_bar(res, main_mode):
    """The main path's speedup over the plain FP32 path at one stated bar
    both meet: the looser of the two stated bars, when both measured errors
    are within it."""
    acc = res["accuracy"]
    if main_mode not in acc or "fp32" not in acc:
        return None
    bar = max(acc[main_mode]["stated_bar"], acc["fp32"]["stated_bar"])
    worst = {m: max(acc[m]["value"], acc[m]["gradient"], acc[m]["laplacian"])
             for m in (main_mode, "fp32")}
    return {"bar": bar, "measured_max": worst, "both_meet": all(v <= bar for v in worst.values()),
            "speedup": res["fp32_path"]["ms_per_step"] / res["ms_per_step"]}


def run_reference(args, rank, world):
    from paper_2512_16677_gb300 import synth
    if rank != 0:
        return None
    mol = synth.make_config(2)
    cores = host_cores()
    n = 48 * cores          # per step: 48 points on each host core
    for _ in range(args.warmup):
        oracle_parallel(mol, mol.points[:n], cores)
    times = []
    used = cores
    for i in range(args.steps):
        # each step: a bounded sample of the workload's points
        start = (i * n) % mol.point_num
        pts = mol.points[start:start + n]
        dt, used = oracle_parallel(mol, pts, cores)
        times.append(dt)
    tot = sum(times)
    value = n * mol.mo_num * args.steps / tot
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "mode": "oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"{n} points per step of the workload, "
                                       f"48 per thread on {used} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    from paper_2512_16677_gb300 import buildlib
    if rank == 0 or world == 1:
        buildlib.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    res, mol, gpu_w0 = run_ours(args, rank, world, local_rank)
    samples = res.pop("_accuracy_samples", {})
    if rank == 0:
        if not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(mol, gpu_w0)
            res["accuracy"] = accuracy(mol, samples, args.mode)
            if res.get("fp32_path") and res["accuracy"]:
                res["speedup_at_common_bar"] = common_bar(res, args.mode)
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
