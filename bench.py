"""Benchmark of the SR-CPM electrode-charge hot path on GB300.

Metric: charge solves/s at 1e-6 relative residual & E-build s.  One step is one pass of
the whole path over one synthetic frame of the precision workload (two graphene sheets
of 40 x 40 cells, 12,800 electrode atoms, 2,000 ions, 98.4 x 170.4 x 90 A box):
k-vector table, structure-factor operand, E = A A^T with the fused real-space terms,
PCG-DC preconditioner, E d' = 1, electrolyte potential b, PCG to 1e-6, neutralisation.
`value` counts solved frames per second over those whole steps; the E-build time and
the solve-only rate are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank is a replica on its own frames (weak scaling): the path has no
data exchange between frames, so the only collectives are the timing barrier and max.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2111_06704_gb300 import workloads as wl  # noqa: E402

METRIC = "charge solves/s at 1e-6 rel. residual & E-build s, vs plain FP64 PCG same GPU"
TOL = 1e-6
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
SMS = 152
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cells", type=int, default=40, help="cells per sheet edge (40: 12,800 atoms)")
    ap.add_argument("--ions", type=int, default=2000)
    ap.add_argument("--precision", choices=["bf16x6", "fp32", "fp64"], default="bf16x6")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------ multi-rank

def max_over_ranks(value: float, world: int) -> float:
    """The slowest rank's time (the job's time); a no-op on one rank."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------ the workload

def make_workload(cells: int, n_ion: int, rank: int):
    el = wl.two_sheet_electrode(cells, cells)
    rng = np.random.default_rng(wl.seed_for(2, rank))
    ions, q = wl.random_ions(rng, n_ion // 2, n_ion // 2, el.box, min_sep=2.5)
    return el, ions[None], q[None]


def kspace_count(box, g=wl.G_EWALD, eps=wl.KSPACE_EPS):
    """Number of half-space k-vectors (same rule as the library's table)."""
    import math
    kc = 2 * g * math.sqrt(math.log(1 / eps))
    lx, ly, lz = box
    hm, km, lm = (int(math.floor(kc * L / (2 * math.pi))) for L in (lx, ly, lz))
    h, k, l = np.meshgrid(np.arange(0, hm + 1), np.arange(-km, km + 1), np.arange(-lm, lm + 1),
                          indexing="ij")
    half = (h > 0) | ((h == 0) & (k > 0)) | ((h == 0) & (k == 0) & (l > 0))
    k2 = (2 * math.pi * h / lx) ** 2 + (2 * math.pi * k / ly) ** 2 + (2 * math.pi * l / lz) ** 2
    return int(np.count_nonzero(half & (k2 <= kc * kc)))


# ------------------------------------------------------------------- the oracle on CPU

def oracle_sample(el, ions, q, n_rows=1, lu_n=2048):
    """Times the FP64 oracle on a bounded sample of one step and scales it to the whole
    step: rows of E and of b^sol by direct sums (scaled by N), a dense bordered solve at
    lu_n (scaled by N^3).  Returns (seconds per full step estimate, description)."""
    from oracle import ewald as ew
    from oracle import solve as sv
    n = el.n
    rows = el.xyz[:n_rows]
    t0 = time.perf_counter()
    others = el.xyz[n_rows:]  # the rows' own r = 0 terms are the diagonal case
    a_ij = ew.mix_alpha(el.alpha[:n_rows, None], el.alpha[None, n_rows:])
    ew.real_space_pairs(rows, others, a_ij, el.box, wl.G_EWALD, wl.RCUT_REAL, same_set=False)
    ew.kspace_pairs(rows, el.xyz, el.box, wl.G_EWALD, wl.KSPACE_EPS)
    t_e = time.perf_counter() - t0
    t0 = time.perf_counter()
    ew.electrolyte_potential(rows, el.alpha[:n_rows], ions[0], q[0], el.box, wl.G_EWALD,
                             wl.RCUT_REAL)
    t_b = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    m = rng.standard_normal((lu_n, lu_n))
    m = m @ m.T / lu_n + np.eye(lu_n)
    t0 = time.perf_counter()
    sv.solve_bordered(m, rng.standard_normal(lu_n), 0.0)
    t_lu = time.perf_counter() - t0
    est = (t_e + t_b) * n / n_rows + t_lu * (n / lu_n) ** 3
    desc = (f"{n_rows} row(s) of E and of b^sol by direct FP64 sums scaled by N={n}, "
            f"bordered LU at N={lu_n} scaled by (N/{lu_n})^3")
    return est, desc


def run_reference(args, rank, world):
    """--impl reference: the FP64 CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return
    el, ions, q = make_workload(args.cells, args.ions, 0)
    for _ in range(args.warmup):
        oracle_sample(el, ions, q)
    times = []
    desc = ""
    for _ in range(args.steps):
        t0 = time.perf_counter()
        est, desc = oracle_sample(el, ions, q)
        times.append(est)
    sec = statistics.mean(times)
    value = 1.0 / sec
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"two-sheet graphene N={el.n}, {args.ions} ions, one frame",
                   "electrode_atoms": el.n, "ions": args.ions},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- our CUDA path

def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2111_06704_gb300 import cpm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    el, ions, q = make_workload(args.cells, args.ions, rank)
    n = el.n
    prec = {"fp32": cpm.CPM_PREC_FP32, "fp64": cpm.CPM_PREC_FP64,
            "bf16x6": cpm.CPM_PREC_BF16X6}[args.precision]
    ctx = cpm.Context(el.box, stream=stream.cuda_stream, precision=prec,
                      precond=cpm.CPM_PRECOND_DC)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    xyz, alpha, ion_xyz, ion_q, chi = t(el.xyz), t(el.alpha), t(ions), t(q), t(el.chi)
    b = torch.empty((1, n), dtype=torch.float64, device=dev)
    qs = torch.empty(1, dtype=torch.float64, device=dev)
    qq = torch.zeros((1, n), dtype=torch.float64, device=dev)
    info = {"kspace_ms": [], "tc_ms": [], "iters": [], "relres": []}

    def step():
        ctx.cpm_build_E(xyz, alpha)
        ctx.cpm_potential(ion_xyz, ion_q, chi, b, qs)
        _, it, rel = ctx.cpm_solve(b, qq, tol=TOL, maxit=2000)
        ctx.cpm_neutralize(qq, qs)
        inf = ctx.cpm_get_info()
        info["kspace_ms"].append(inf["t_kspace_ms"])
        info["tc_ms"].append(inf["t_tc_ms"])
        info["head_cols"] = inf["head_cols"]
        info["iters"].append(int(it[0]))
        info["relres"].append(float(rel[0]))

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        info = {k: ([] if isinstance(v, list) else v) for k, v in info.items()}
        if world > 1:
            dist.barrier()
        launches0 = ctx.cpm_get_info()["launches"]
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clocks:
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(args.steps):
                step()
            ev1.record(stream)
            torch.cuda.synchronize()
        launches = ctx.cpm_get_info()["launches"] - launches0
        ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world)
        if world > 1:
            dist.barrier()

        # solve-only rate: potential + PCG + neutralise with E already built
        ev0.record(stream)
        reps = 5
        for _ in range(reps):
            ctx.cpm_potential(ion_xyz, ion_q, chi, b, qs)
            ctx.cpm_solve(b, qq, tol=TOL, maxit=2000)
            ctx.cpm_neutralize(qq, qs)
        ev1.record(stream)
        torch.cuda.synchronize()
        solve_ms = ev0.elapsed_time(ev1) / reps

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        xyz_h, alpha_h, chi_h = el.xyz.copy(), el.alpha.copy(), el.chi.copy()
        ions_h, q_h = ions.copy(), q.copy()

        def step_host():
            ctx.cpm_build_E(xyz_h, alpha_h)
            bh, qsh = ctx.cpm_potential(ions_h, q_h, chi_h)
            qh, _, _ = ctx.cpm_solve(bh, tol=TOL, maxit=2000)
            ctx.cpm_neutralize(qh, qsh)
            return qh

        step_host()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
        h2d = 8 * (n * 3 + n + ions.size + q.size + n + n + n + 1)
        d2h = 8 * (n + 1 + n + n)
        e2e = {"value": world / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    if rank != 0:
        return
    peaks, src = measured_peaks()
    m = kspace_count(el.box)
    kspace_ms = statistics.mean(info["kspace_ms"])
    # algorithmic FLOPs of the k-space GEMM: lower triangle incl. diagonal, 2M columns
    flops = 2.0 * (n * (n + 1) / 2) * (2 * m)
    clk = clocks.summary()
    sm_mhz = clk.get("sm_max_mhz") or 2070.0
    esz = 8 if args.precision == "fp64" else 4
    if args.precision == "bf16x6":
        # the tensor-core tail kernel alone: lower-triangle tiles, tail columns, six BF16
        # products per term (the FP64 head kernel is timed apart in e_build_s)
        tc_ms = statistics.mean(info["tc_ms"])
        nt = (n + 127) // 128
        tail_cols = 2 * ((m + 63) // 64 * 64) - info["head_cols"]
        tc_flops = 6 * 2.0 * (nt * (nt + 1) / 2) * 128 * 128 * tail_cols
        algo_flops = 6 * 2.0 * (n * (n + 1) / 2) * tail_cols
        bf16_peak = peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"])
        roof = {"bound": "tensor", "achieved": algo_flops / (tc_ms * 1e-3) / 1e12,
                "peak": bf16_peak, "unit": "TFLOP/s",
                "kernel": "k_ek_tc (tcgen05 BF16x6 k-space GEMM, TMEM two-sum accumulation)",
                "peak_source": f"{src} bf16_tflops (burst)",
                "issued_tflops": tc_flops / (tc_ms * 1e-3) / 1e12,
                "fp32_accurate_tflops": algo_flops / 6 / (tc_ms * 1e-3) / 1e12}
    elif args.precision == "fp32":
        peak = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops / (kspace_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "kernel": "k_ek_simt<float> (k-space GEMM + fused epilogue)",
                "peak_source": f"derived: {SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                               f"{sm_mhz:.0f} MHz"}
    else:
        peak = SMS * 64 * 2 * sm_mhz * 1e6 / 1e12 / 32.0
        roof = {"bound": "alu", "achieved": flops / (kspace_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "kernel": "k_ek_simt<double>",
                "peak_source": "derived FP64 rate"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    value = world * 1000.0 / ms
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "bf16x6": "bf16x6 (f32-accurate)"}[args.precision], "data": "synthetic",
        "config": {"workload": f"two-sheet graphene N={n}, {args.ions} ions, one frame per "
                               f"step incl. full E/P/d build",
                   "electrode_atoms": n, "ions": args.ions, "kvectors": m,
                   "l2": "working set > L2 (E %.0f MB, A %.1f GB)" % (
                       n * n * esz / 1e6,
                       n * 2 * m * esz / 1e9),
                   "tol": TOL, "precond": "PCG-DC (g=0.083, r_cut=8)"},
        "e_build_s": kspace_ms / 1e3,
        "solve_only": {"value": 1000.0 / solve_ms, "unit": "solves/s",
                       "iters": statistics.median(info["iters"])},
        "relres": max(info["relres"]),
        "roofline": roof,
        "peaks": {"source": src},
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        est, desc = oracle_sample(el, ions, q)
        line["cpu_baseline"] = {"value": 1.0 / est, "unit": "solves/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": desc}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
