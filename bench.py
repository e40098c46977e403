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
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 10 for the default workload, whose 140 ms "
                         "steps then span enough clock samples; 3 otherwise)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cells", type=int, default=40, help="cells per sheet edge (40: 12,800 atoms)")
    ap.add_argument("--ions", type=int, default=2000)
    ap.add_argument("--precision", choices=["bf16x6", "fp32", "fp64"], default="bf16x6")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=["scale-point", "precision", "batch", "learned",
                                           "matvec", "scale", "scale-learned", "build",
                                           "potential"],
                    default="scale-point")
    ap.add_argument("--rhs", type=int, default=1,
                    help="directions per matvec (matvec workload), frames per step (scale)")
    ap.add_argument("--ragged", type=int, default=32,
                    help="ragged systems in the batch workload (0: skip that part)")
    ap.add_argument("--train-frames", type=int, default=20000)
    ap.add_argument("--heldout-frames", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--frames", type=int, default=256, help="frames per batch (batch workload)")
    ap.add_argument("--stack", type=int, nargs=2, default=[90, 52], metavar=("NX", "NY"),
                    help="build workload: cells of each of the six stacked sheets (90 52: the "
                         "scale point's electrode)")
    ap.add_argument("--sheets", type=int, default=6,
                    help="build workload: stacked sheets (6: the scale point's electrode)")
    ap.add_argument("--stream", action="store_true",
                    help="matvec workload: time the streamed 16-column matvec inside a PCG solve "
                         "of --rhs random right-hand sides instead of cpm_apply_E")
    ap.add_argument("--matrix-path", action="store_true",
                    help="batch workload: also time the matrix path (S formed once, q = S b)")
    ap.add_argument("--baseline-frames", type=int, default=None,
                    help="frames timed for the per-frame FP64 baseline (default: 16 for the "
                         "batch workload, 2 at the scale point)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = {"scale-point": 10, "precision": 10}.get(args.workload, 3)
    if args.baseline_frames is None:
        args.baseline_frames = 2 if args.workload == "scale-point" else 16
    return args


def stream_traffic():
    """DRAM bytes (read + write) per element of E of one k_matvec_stream launch, read from
    the committed summary of that kernel's ncu capture (a 25,992-atom case, 16 columns);
    the bench scales it to a full launch by N^2.  (None, note) when the summary is absent."""
    import re
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles",
                        "k_matvec_stream_N25992.md")
    try:
        text = open(path).read()
    except OSError:
        return None, "no capture summary"
    m = re.search(r"DRAM bytes per element of E \(read \+ write\)[^|]*\|\s*([0-9.]+)", text)
    if not m:
        return None, "no traffic figure in the capture summary"
    return float(m.group(1)), ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                               "launch at N=25,992 (profiles/k_matvec_stream_N25992.md), "
                               "per element of E, times N^2")


def tail_traffic():
    """DRAM bytes (read + write) per tile and tail K-block of the tensor-core tail, read from
    the committed summary of its ncu capture (a reduced scale-point electrode); the bench
    scales it by tiles x K-blocks.  (None, note) when the summary is absent."""
    import re
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles",
                        "k_ek_strip_stacked_N8869.md")
    try:
        text = open(path).read()
    except OSError:
        return None, "no capture summary"
    m = re.search(r"\|\s*DRAM bytes per tile and K-block\s*\|\s*([0-9,]+)", text)
    if not m:
        return None, "no traffic figure in the capture summary"
    return float(m.group(1).replace(",", "")), (
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of both tile launches at N=8,869 "
        "(profiles/k_ek_strip_stacked_N8869.md), per tile and K-block, times tiles x K-blocks")


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
    return est, t_e + t_b + t_lu, desc


def oracle_small_cell():
    """The FP64 oracle timed as it stands on one whole charge solve of the 512-atom cell
    with 200 ions: E by the direct pairwise sums (the build), then b^sol by direct sums and
    the bordered dense solve (the charge solve).  Returns (build s, solve s)."""
    from oracle import ewald as ew
    from oracle import solve as sv
    work = wl.small_cell()
    el, io = work.electrode, work.electrolyte
    t0 = time.perf_counter()
    e = ew.interaction_matrix(el.xyz, el.alpha, el.box, wl.G_EWALD, wl.RCUT_REAL,
                              wl.KSPACE_EPS, True)
    t1 = time.perf_counter()
    bsol = ew.electrolyte_potential(el.xyz, el.alpha, io.xyz[0], io.q[0], el.box, wl.G_EWALD,
                                    wl.RCUT_REAL, wl.KSPACE_EPS, True)
    sv.solve_bordered(e, ew.rhs_volts(el.chi, bsol) / ew.KE, float(io.q[0].sum()))
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


def oracle_scale_sample(el, ion_xyz, ion_q, g, rc, rows=16, k_sample=512, tri_n=3072):
    """A bounded sample of the oracle's charge solve at the scale point, with E built and
    factored (the build alone, 91 GB and ~4e14 FLOP of FP64 Cholesky, is out of reach on
    the host): the reciprocal part of b^sol through the ions' structure factors over
    k_sample of the table's k-vectors, the real-space part for `rows` electrode atoms
    against every ion, and the two triangular solves of a factored E at tri_n; each part
    scaled to the whole (k-vectors, atoms, N^2).  Returns (seconds per solve, text)."""
    import scipy.linalg as sla

    from oracle import ewald as ew
    n, n_ion = el.n, ion_q.shape[0]
    _, kvec, w = ew.kvectors(el.box, g, wl.KSPACE_EPS)
    m = kvec.shape[0]
    kc = kvec[:k_sample]
    t0 = time.perf_counter()
    phi = ion_xyz @ kc.T
    re, im = np.cos(phi).T @ ion_q, np.sin(phi).T @ ion_q
    ph = el.xyz @ kc.T
    _ = np.cos(ph) @ (w[:k_sample] * re) + np.sin(ph) @ (w[:k_sample] * im)
    t_k = (time.perf_counter() - t0) * m / k_sample
    t0 = time.perf_counter()
    ew.real_space_pairs(el.xyz[:rows], ion_xyz, el.alpha[:rows, None], el.box, g, rc,
                        same_set=False)
    t_r = (time.perf_counter() - t0) * n / rows
    rng = np.random.default_rng(0)
    lower = np.tril(rng.standard_normal((tri_n, tri_n))) + tri_n * np.eye(tri_n)
    rhs = rng.standard_normal(tri_n)
    t0 = time.perf_counter()
    y = sla.solve_triangular(lower, rhs, lower=True)
    sla.solve_triangular(lower.T, y, lower=False)
    t_tri = time.perf_counter() - t0
    t_s = t_tri * (n / tri_n) ** 2
    wall = t_k * k_sample / m + t_r * rows / n + t_tri
    desc = (f"oracle at N={n}, {n_ion} ions, E built and factored: b^sol reciprocal part over "
            f"{k_sample} of {m} k-vectors scaled by {m / k_sample:.0f}, real space for {rows} "
            f"atoms scaled by N/{rows}, two triangular solves at N={tri_n} scaled by "
            f"(N/{tri_n})^2")
    return t_k + t_r + t_s, wall, desc


def run_reference(args, rank, world):
    """--impl reference: the FP64 CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return
    if args.workload == "scale-point":
        # the default workload: a bounded sample of the oracle's charge solve at the scale
        # point, per frame (the step's 16 frames are independent solves for the oracle)
        work = wl.scale_point(seed=wl.seed_for(5, 0), rhs=1)
        el, io = work.electrode, work.electrolyte
        sample = lambda: oracle_scale_sample(el, io.xyz[0], io.q[0], SCALE_G, SCALE_RC)
        config = {"workload": SCALE_WORKLOAD.format(n=el.n, ions=io.n_ion, frames=1),
                  "electrode_atoms": el.n, "ions": io.n_ion, "frames_per_step": 1,
                  "g_ewald": SCALE_G, "rcut_real": SCALE_RC}
    else:
        el, ions, q = make_workload(args.cells, args.ions, 0)
        sample = lambda: oracle_sample(el, ions, q)
        config = {"workload": f"two-sheet graphene N={el.n}, {args.ions} ions, one frame",
                  "electrode_atoms": el.n, "ions": args.ions}
    for _ in range(args.warmup):
        sample()
    ests, walls = [], []
    desc = ""
    for _ in range(args.steps):
        est, wall, desc = sample()
        ests.append(est)
        walls.append(wall)
    # each step is the bounded sample itself (its wall time is ms_per_step); the value is
    # the fraction of one solve it covers over that time
    value = 1.0 / statistics.mean(ests)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(walls) * 1e3, "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": desc + "; a step is this sample, a fraction "
                                          f"{statistics.mean(walls) / statistics.mean(ests):.2e} "
                                          "of one solve"},
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
    info = {"kspace_ms": [], "tc_ms": [], "head_ms": [], "light_ms": [], "iters": [], "relres": []}

    def step():
        ctx.cpm_build_E(xyz, alpha)
        ctx.cpm_potential(ion_xyz, ion_q, chi, b, qs)
        _, it, rel = ctx.cpm_solve(b, qq, tol=TOL, maxit=2000)
        ctx.cpm_neutralize(qq, qs)
        inf = ctx.cpm_get_info()
        info["kspace_ms"].append(inf["t_kspace_ms"])
        info["tc_ms"].append(inf["t_tc_ms"])
        info["head_cols"] = inf["head_cols"]
        info["tc_blocks"] = list(inf["tc_blocks"])
        info["tc_blocks_fp8"] = inf["tc_blocks_fp8"]
        info["head_ms"].append(inf["t_head_ms"])
        info["light_ms"].append(inf["t_tc_light_ms"])
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
        # the PCG matvec alone (one column; events inside the library around its launch)
        mv_ms = []
        for _ in range(6):
            ctx.cpm_apply_E(qq, b)
            mv_ms.append(ctx.cpm_get_info()["t_matvec_ms"])
        matvec_ms = statistics.median(mv_ms[1:])

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
    m = cpm.cpm_plan_kspace(el.box)["m"]  # k-vectors of the build's table
    kspace_ms = statistics.mean(info["kspace_ms"])
    # algorithmic FLOPs of the k-space GEMM: lower triangle incl. diagonal, 2M columns
    flops = 2.0 * (n * (n + 1) / 2) * (2 * m)
    clk = clocks.summary()
    sm_mhz = clk.get("sm_max_mhz") or 2070.0
    esz = 8 if args.precision == "fp64" else 4
    if args.precision == "bf16x6":
        # the tensor-core tail kernel alone: lower-triangle tiles over the tail columns,
        # each 64-column K-block with six, three or one BF16 products (weight-bounded
        # schedule); the FP64-accurate head kernel is timed apart and sits in e_build_s
        tc_ms = statistics.mean(info["tc_ms"])
        # 256 x 256 tiles of the lower triangle; a diagonal tile skips its upper-right
        # 128 x 128 quarter
        nt = (n + 255) // 256
        n6, n3, n1 = info["tc_blocks"]
        prod_cols = 64 * (6 * n6 + 3 * n3 + n1)
        tail_cols = 64 * (n6 + n3 + n1)
        tc_flops = 2.0 * (nt * (nt - 1) / 2 + 0.75 * nt) * 256 * 256 * prod_cols
        algo_flops = 2.0 * (n * (n + 1) / 2) * prod_cols
        # the tail runs ~100 ms without a break inside each step: the sustained (power-
        # capped) BF16 rate is its denominator; the burst one is reported beside it
        bf16_peak = peaks.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"])
        burst = peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"])
        roof = {"bound": "tensor", "achieved": algo_flops / (tc_ms * 1e-3) / 1e12,
                "peak": bf16_peak, "unit": "TFLOP/s",
                "kernel": "k_ek_strip<true> + k_ek_strip<false> (tcgen05 k-space GEMM on "
                          "256 x 256 tiles: six BF16 products per heavy K-block, then three or "
                          "one FP16 or one FP8 product of per-block scaled values; two-sum chunk "
                          "drains into per-SM hi/lo scratch)",
                "peak_source": f"{src} bf16_tflops_sustained",
                "frac_of_burst": algo_flops / (tc_ms * 1e-3) / 1e12 / burst,
                "issued_tflops": tc_flops / (tc_ms * 1e-3) / 1e12,
                "fp32_accurate_tflops": 2.0 * (n * (n + 1) / 2) * tail_cols / (tc_ms * 1e-3) / 1e12,
                "k_blocks_6_3_1_products": [n6, n3, n1],
                "k_blocks_fp8": info.get("tc_blocks_fp8"),
                "tc_ms": tc_ms, "light_ms": statistics.mean(info["light_ms"]),
                "head_ms": statistics.mean(info["head_ms"])}
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
    if args.precision == "bf16x6" and n == 12800:
        # DRAM read + write of the two tail launches of one build, from a one-pass ncu
        # launch list of this workload (dram__bytes_read.sum + dram__bytes_write.sum)
        roof["traffic"] = 488.5e9
        roof["traffic_unit"] = "bytes per build (both launches)"
    value = world * 1000.0 / ms
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "bf16x6": "bf16x6+fp16x3+fp8 (f32-accurate)"}[args.precision], "data": "synthetic",
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
        "matvec_roofline": {
            "bound": "hbm", "kernel": "k_matvec (PCG matvec, E streamed once)",
            "achieved": n * ((n + 127) // 128 * 128) * esz / (matvec_ms * 1e-3) / 1e9,
            "peak": peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]), "unit": "GB/s",
            "frac": n * ((n + 127) // 128 * 128) * esz / (matvec_ms * 1e-3) / 1e9
            / peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]),
            "ms": matvec_ms, "bytes_per_launch": n * ((n + 127) // 128 * 128) * esz},
        "peaks": {"source": src},
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        est, _, desc = oracle_sample(el, ions, q)
        line["cpu_baseline"] = {"value": 1.0 / est, "unit": "solves/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": desc}
    print(json.dumps(line), flush=True)


def run_matvec(args, rank, world, local_rank):
    """The PCG matvec alone: E of the `--cells` two-sheet electrode (FP32 storage) applied
    to `--rhs` directions per call through cpm_apply_E, timed by CUDA events inside the
    library around its matvec launches.  The matvec streams E whatever its entries are,
    so the k-space cutoff is loosened to 1e-3 to keep the build (and the device memory
    a counter capture saves and restores) small."""
    import torch

    from paper_2111_06704_gb300 import cpm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    el = wl.two_sheet_electrode(args.cells, args.cells)
    n = el.n
    ctx = cpm.Context(el.box, precision=cpm.CPM_PREC_FP32, kspace_eps=1e-3)
    ctx.cpm_build_E(el.xyz, el.alpha)
    rng = np.random.default_rng(wl.seed_for(2, rank))
    p = torch.tensor(rng.standard_normal((args.rhs, n)), device=dev)
    q = torch.empty_like(p)

    def once():
        if args.stream:  # the PCG iterations' streamed matvec, per launch
            q.zero_()
            _, it, _ = ctx.cpm_solve(p, q, tol=1e-6, maxit=500)
            inf = ctx.cpm_get_info()
            return inf["t_solve_matvec_ms"] / max(1, int(np.max(it)))
        ctx.cpm_apply_E(p, q)
        return ctx.cpm_get_info()["t_matvec_ms"]

    for _ in range(args.warmup):
        once()
    ms = []
    with ClockSampler(local_rank) as clocks:
        for _ in range(args.steps):
            ms.append(once())
    ms = max_over_ranks(statistics.median(ms), world)
    if rank != 0:
        return
    e_bytes = n * ((n + 127) // 128 * 128) * 4
    peak = measured_peaks()[0].get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    gbs = world * e_bytes / (ms * 1e-3) / 1e9
    line = {"metric": "PCG matvec E-streaming rate", "value": gbs, "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"matvec: two-sheet graphene N={n}, {args.rhs} right-hand "
                                   f"side(s) per pass, E {e_bytes / 1e6:.0f} MB"
                                   + (", the streamed matvec of PCG iterations"
                                      if args.stream else ""),
                       "l2": "E larger than L2" if e_bytes > 129e6 else "E fits in L2"},
            "roofline": {"bound": "hbm", "achieved": gbs / world, "peak": peak, "unit": "GB/s",
                         "frac": gbs / world / peak, "traffic": None},
            "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)


def run_potential(args, rank, world, local_rank):
    """cpm_potential alone: b of `--frames` frames of `--ions` ions (Gaussian perturbations
    of one seeded frame) on the `--cells` two-sheet electrode, timed with CUDA events, with
    the library's phase times (ion structure factors, k-space, real space).  The k-space
    cutoff is loosened to 1e-3, which keeps the build and its device memory small; the
    real-space sums, which dominate at this size, are those of the default parameters."""
    import torch

    from paper_2111_06704_gb300 import cpm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    el, ions, q = make_workload(args.cells, args.ions, rank)
    frames = max(1, min(args.frames, 64))
    rng = np.random.default_rng(wl.seed_for(2, 50 + rank))
    xyz = wl.perturb_frames(rng, ions[0], frames, 0.5, el.box)
    qi = np.broadcast_to(q[0], (frames, q.shape[1])).copy()
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    ctx = cpm.Context(el.box, stream=stream.cuda_stream, kspace_eps=1e-3)
    ctx.cpm_build_E(t(el.xyz), t(el.alpha))
    x, qq, chi = t(xyz), t(qi), t(el.chi)
    b = torch.empty((frames, el.n), dtype=torch.float64, device=dev)
    qs = torch.empty(frames, dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        ctx.cpm_potential(x, qq, chi, b, qs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts, parts = [], []
    with ClockSampler(local_rank) as clocks:
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0.record(stream)
            ctx.cpm_potential(x, qq, chi, b, qs)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            inf = ctx.cpm_get_info()
            parts.append((inf["t_pot_sf_ms"], inf["t_pot_kspace_ms"], inf["t_pot_real_ms"]))
    ms = max_over_ranks(statistics.median(ts), world)
    if rank != 0:
        return
    line = {"metric": "potential frames/s", "value": world * frames * 1000.0 / ms,
            "unit": "frames/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 b (float-pair and float sums inside)",
            "data": "synthetic",
            "config": {"workload": f"potential: two-sheet graphene N={el.n}, {frames} frames of "
                                   f"{args.ions} ions, k-space cutoff 1e-3",
                       "kvectors": inf["m"]},
            "phase_ms": {"ion_structure_factors": parts[-1][0], "kspace": parts[-1][1],
                         "real_space_and_finish": parts[-1][2]},
            "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)


def run_build(args, rank, world, local_rank):
    """The E build alone (cpm_build_E: operand, head, tensor-core tail, PCG-DC, d) of the
    scale point's electrode or a smaller one of the same kind (six stacked sheets of
    --stack NX NY cells with 5% pinholes, g = 0.15, r_c = 24), timed with CUDA events; the
    tail's method-FLOP roofline against the sustained BF16 rate."""
    import torch

    from paper_2111_06704_gb300 import cpm

    torch.cuda.set_device(local_rank)
    rng = np.random.default_rng(wl.seed_for(5, rank))
    el = wl.stacked_electrode(rng, nx=args.stack[0], ny=args.stack[1], sheets=args.sheets)
    n = el.n
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    ctx = cpm.Context(el.box, stream=stream.cuda_stream, g_ewald=SCALE_G, rcut_real=SCALE_RC)
    for _ in range(args.warmup):
        ctx.cpm_build_E(el.xyz, el.alpha)
    ts, tcs = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clocks:
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0.record(stream)
            ctx.cpm_build_E(el.xyz, el.alpha)
            e1.record(stream)
            torch.cuda.synchronize()
            inf = ctx.cpm_get_info()
            ts.append(e0.elapsed_time(e1))
            tcs.append(inf["t_tc_ms"])
    ms = max_over_ranks(statistics.median(ts), world)
    if rank != 0:
        return
    peaks, src = measured_peaks()
    sustained = peaks.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"])
    n6, n3, n1 = inf["tc_blocks"]
    tail_cols = 64 * (n6 + n3 + n1)
    tc_ms = statistics.median(tcs)
    achieved = 2.0 * (n * (n + 1) / 2) * tail_cols / (tc_ms * 1e-3) / 1e12
    line = {"metric": "E builds/s", "value": world * 1000.0 / ms, "unit": "builds/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x6+fp16x3+fp8 (f32-accurate E)", "data": "synthetic",
            "config": {"workload": f"E build: {args.sheets} stacked {args.stack[0]} x "
                                   f"{args.stack[1]}-cell "
                                   f"graphene sheets with pinholes, N={n}, g={SCALE_G}, "
                                   f"r_c={SCALE_RC}", "electrode_atoms": n,
                       "kvectors": inf["m"]},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": sustained,
                         "unit": "TFLOP/s", "frac": achieved / sustained, "traffic": None,
                         "kernel": "k_ek_strip (tcgen05 k-space tail)",
                         "work": "method FLOPs: N(N+1)/2 x 2 x tail operand columns "
                                 f"({tail_cols})", "tc_ms": tc_ms,
                         "peak_source": f"{src} bf16_tflops_sustained (of measured)"},
            "build_ms": {"kspace": inf["t_kspace_ms"], "head": inf["t_head_ms"],
                         "tensor_core": tc_ms, "precond": inf["t_precond_ms"],
                         "d_solve": inf["t_dsolve_ms"]},
            "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)


def run_scale(args, rank, world, local_rank):
    """Scale point: six stacked graphene sheets with 5% pinholes (~106,600 atoms, dense E
    45 GB) and 20,000 ions, `--rhs` perturbed frames per step.  The structure-factor
    operand (79 GB) is not kept: the build streams it in k-windows and the potential sums
    its k-space part directly.  g = 0.15 1/A with r_c = 24 A (E does not depend on g).
    The build is timed once; a step is the potential of every frame, one multi-RHS PCG-DC
    solve and the neutralisation."""
    import torch

    from paper_2111_06704_gb300 import cpm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    work = wl.scale_point(seed=wl.seed_for(5, rank), rhs=args.rhs)
    el, io = work.electrode, work.electrolyte
    n, F = el.n, io.frames
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    xyz, alpha, chi, ion_xyz, ion_q = t(el.xyz), t(el.alpha), t(el.chi), t(io.xyz), t(io.q)
    ctx = cpm.Context(el.box, stream=stream.cuda_stream, g_ewald=0.15, rcut_real=24.0)
    b = torch.empty((F, n), dtype=torch.float64, device=dev)
    qs = torch.empty(F, dtype=torch.float64, device=dev)
    q = torch.zeros((F, n), dtype=torch.float64, device=dev)
    iters = []

    def step():
        ctx.cpm_potential(ion_xyz, ion_q, chi, b, qs)
        q.zero_()
        _, it, _ = ctx.cpm_solve(b, q, tol=TOL, maxit=3000)
        ctx.cpm_neutralize(q, qs)
        iters.append(float(np.mean(it)))

    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.cpm_build_E(xyz, alpha)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        inf = ctx.cpm_get_info()
        for _ in range(args.warmup):
            step()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clocks:
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(args.steps):
                step()
            ev1.record(stream)
            torch.cuda.synchronize()
        ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world)
        mv = []
        for _ in range(4):
            ctx.cpm_apply_E(q[:1], b[:1])
            mv.append(ctx.cpm_get_info()["t_matvec_ms"])
        mv_ms = statistics.median(mv[1:])
    if rank != 0:
        return
    e_bytes = n * ((n + 127) // 128 * 128) * 4
    peak = measured_peaks()[0].get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    line = {
        "metric": METRIC, "value": world * F * 1000.0 / ms, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x6+fp16x3+fp8 (f32-accurate)", "data": "synthetic",
        "config": {"workload": f"scale point: six stacked graphene sheets with pinholes, "
                               f"N={n}, {io.n_ion} ions, {F} frames per step (build once)",
                   "electrode_atoms": n, "ions": io.n_ion, "rhs": F, "tol": TOL,
                   "g_ewald": 0.15, "rcut_real": 24.0, "kvectors": inf["m"],
                   "l2": f"E {e_bytes / 1e9:.1f} GB, streamed once per PCG iteration"},
        "e_build_s": build_s,
        "build_ms": {"kspace": inf["t_kspace_ms"], "tensor_core": inf["t_tc_ms"],
                     "head": inf["t_head_ms"], "precond": inf["t_precond_ms"],
                     "d_solve": inf["t_dsolve_ms"]},
        "mean_iters": statistics.mean(iters),
        "matvec_roofline": {"bound": "hbm", "achieved": e_bytes / (mv_ms * 1e-3) / 1e9,
                            "peak": peak, "unit": "GB/s",
                            "frac": e_bytes / (mv_ms * 1e-3) / 1e9 / peak, "ms": mv_ms},
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


def run_batch(args, rank, world, local_rank):
    """Batching form: the 512-atom electrode, `--frames` frames of 2,000 ions (Gaussian
    perturbations of one base frame) solved as one multi-right-hand-side PCG, against the
    plain per-frame path on the same GPU (FP64 E, FP64 Jacobi PCG, one frame per call)."""
    import torch

    from paper_2111_06704_gb300 import cpm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    work = wl.frame_batch(frames=args.frames, seed=wl.seed_for(3, rank))
    el, io = work.electrode, work.electrolyte
    n, F = el.n, io.frames
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    xyz, alpha, chi, ion_xyz, ion_q = t(el.xyz), t(el.alpha), t(el.chi), t(io.xyz), t(io.q)
    ctx = cpm.Context(el.box, stream=stream.cuda_stream, precision=cpm.CPM_PREC_BF16X6,
                      precond=cpm.CPM_PRECOND_DC)
    base = cpm.Context(el.box, stream=stream.cuda_stream, precision=cpm.CPM_PREC_FP64,
                       precond=cpm.CPM_PRECOND_JACOBI)
    b = torch.empty((F, n), dtype=torch.float64, device=dev)
    qs = torch.empty(F, dtype=torch.float64, device=dev)
    q = torch.zeros((F, n), dtype=torch.float64, device=dev)
    iters = []

    def step():
        ctx.cpm_build_E(xyz, alpha)
        ctx.cpm_potential(ion_xyz, ion_q, chi, b, qs)
        _, it, _ = ctx.cpm_solve(b, q, tol=TOL, maxit=2000)
        ctx.cpm_neutralize(q, qs)
        iters.append(float(np.mean(it)))

    def timed(fn, reps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        launches0 = ctx.cpm_get_info()["launches"]
        with ClockSampler(local_rank) as clocks:
            ms = max_over_ranks(timed(step, args.steps), world)
        launches = ctx.cpm_get_info()["launches"] - launches0
        solve_ms = timed(lambda: (ctx.cpm_solve(b, q, tol=TOL, maxit=2000),
                                  ctx.cpm_neutralize(q, qs)), 3)
        pot_ms = timed(lambda: ctx.cpm_potential(ion_xyz, ion_q, chi, b, qs), 3)
        matrix = None
        if args.matrix_path:
            # the matrix path on the same E: S formed once, then one product per batch
            build_ms = timed(lambda: ctx.cpm_smatrix_build(tol=1e-10, maxit=2000), 1)
            qm = torch.empty((F, n), dtype=torch.float64, device=dev)
            mat_ms = timed(lambda: ctx.cpm_smatrix_charges(b, qs, qm), 3)
            matrix = {"s_build_ms": build_ms,
                      "charges": {"value": F * 1000.0 / mat_ms, "unit": "solves/s",
                                  "what": "cpm_smatrix_charges alone (b given)"},
                      "with_b": {"value": F * 1000.0 / (mat_ms + pot_ms), "unit": "solves/s"},
                      "max_rel_diff_vs_pcg": float((qm - q).abs().max() / q.abs().max())}

        # plain per-frame FP64 Jacobi PCG on the same GPU, zero and previous-step guesses
        base.cpm_build_E(xyz, alpha)
        nb = min(F, args.baseline_frames)
        b1 = torch.empty((1, n), dtype=torch.float64, device=dev)
        q1 = torch.zeros((1, n), dtype=torch.float64, device=dev)
        qs1 = torch.empty(1, dtype=torch.float64, device=dev)
        it_base = []

        def base_frames(guess):
            for f in range(nb):
                base.cpm_potential(ion_xyz[f:f + 1], ion_q[f:f + 1], chi, b1, qs1)
                if not guess:
                    q1.zero_()
                _, it, _ = base.cpm_solve(b1, q1, use_guess=guess, tol=TOL, maxit=5000)
                base.cpm_neutralize(q1, qs1)
                it_base.append(int(it[0]))

        base_ms = timed(lambda: base_frames(False), 1) / nb
        base_it = float(np.mean(it_base))
        it_base.clear()
        base_prev_ms = timed(lambda: base_frames(True), 1) / nb
        base_solve_ms = timed(lambda: [(base.cpm_solve(b1, q1, tol=TOL, maxit=5000),
                                        base.cpm_neutralize(q1, qs1)) for _ in range(nb)], 1) / nb
        ragged = run_ragged(args, rank, dev, stream, timed) if args.ragged > 0 else None
    if rank != 0:
        return
    value = world * F * 1000.0 / ms
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x6+fp16x3+fp8 (f32-accurate)", "data": "synthetic",
        "config": {"workload": f"batching form: two-sheet graphene N={n}, {F} frames x "
                               f"{io.n_ion} ions per step incl. E/P/d build",
                   "frames": F, "ions": io.n_ion, "tol": TOL,
                   "l2": "E (1 MB) is L2-resident; batched frames share each pass over it"},
        "solve_only": {"value": F * 1000.0 / solve_ms, "unit": "solves/s",
                       "mean_iters": statistics.mean(iters)},
        "potential_ms_per_batch": pot_ms,
        "baseline_fp64_per_frame": {
            "value": 1000.0 / base_ms, "unit": "solves/s", "mean_iters": base_it,
            "prev_step_guess_value": 1000.0 / base_prev_ms,
            "solve_only_value": 1000.0 / base_solve_ms, "frames_timed": nb,
            "what": "FP64 E, FP64 Jacobi PCG, cpm_potential + cpm_solve + cpm_neutralize "
                    "one frame per call"},
        "speedup_vs_fp64_per_frame": {"with_b": (F * 1000.0 / ms) / (1000.0 / base_ms),
                                      "solve_only": (F / solve_ms) / (1.0 / base_solve_ms)},
        "clocks": clocks.summary(),
        "gpu_launches": launches,
    }
    if ragged is not None:
        line["ragged"] = ragged
    if matrix is not None:
        line["matrix_path"] = matrix
    print(json.dumps(line), flush=True)


def run_ragged(args, rank, dev, stream, timed):
    """The ragged part of the batching form: `--ragged` independent two-sheet systems with
    electrode counts drawn uniformly in [500, 8000] (one frame each), built once; timed: the
    potentials, then one batched PCG over all systems plus the batched neutralisation,
    against the same systems solved one context at a time."""
    import torch

    from paper_2111_06704_gb300 import cpm

    works = wl.ragged_systems(count=args.ragged, n_lo=500, n_hi=8000,
                              seed=wl.seed_for(3, 100 + rank))
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    ctxs, ins = [], []
    for w in works:
        el, io = w.electrode, w.electrolyte
        c = cpm.Context(el.box, stream=stream.cuda_stream, precision=cpm.CPM_PREC_BF16X6,
                        precond=cpm.CPM_PRECOND_DC)
        c.cpm_build_E(t(el.xyz), t(el.alpha))
        ctxs.append(c)
        ins.append((t(io.xyz), t(io.q), t(el.chi)))
    build_s = time.perf_counter() - t0
    sizes = [c.n for c in ctxs]
    tot = sum(sizes)
    b = torch.empty(tot, dtype=torch.float64, device=dev)
    q = torch.zeros(tot, dtype=torch.float64, device=dev)
    qs = torch.empty(len(ctxs), dtype=torch.float64, device=dev)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    batch = cpm.Batch(ctxs)
    its = {}

    def potentials():
        for k, (c, (x, qi, chi)) in enumerate(zip(ctxs, ins)):
            c.cpm_potential(x, qi, chi, b[offs[k]:offs[k + 1]].view(1, -1), qs[k:k + 1])

    def batched(with_b=True):
        if with_b:
            potentials()
        q.zero_()
        _, it, _ = batch.solve(b, q, tol=TOL, maxit=2000)
        batch.neutralize(q, qs)
        its["batch"] = float(np.mean(it))

    def one_by_one(with_b=True):
        if with_b:
            potentials()
        q.zero_()
        it_all = []
        for k, c in enumerate(ctxs):
            qk = q[offs[k]:offs[k + 1]].view(1, -1)
            _, it, _ = c.cpm_solve(b[offs[k]:offs[k + 1]].view(1, -1), qk, tol=TOL, maxit=2000)
            c.cpm_neutralize(qk, qs[k:k + 1])
            it_all.append(int(it[0]))
        its["single"] = float(np.mean(it_all))

    batched()
    one_by_one()
    ms_batch = timed(batched, 2)
    ms_single = timed(one_by_one, 2)
    pot_ms = timed(potentials, 2)
    ms_batch_solve = timed(lambda: batched(False), 2)
    ms_single_solve = timed(lambda: one_by_one(False), 2)
    out = {"systems": len(ctxs), "atoms_min": min(sizes), "atoms_max": max(sizes),
           "atoms_total": tot, "build_s_all": build_s,
           "batched": {"value": len(ctxs) * 1000.0 / ms_batch, "unit": "solves/s",
                       "ms": ms_batch, "mean_iters": its["batch"]},
           "one_context_at_a_time": {"value": len(ctxs) * 1000.0 / ms_single,
                                     "unit": "solves/s", "ms": ms_single,
                                     "mean_iters": its["single"]},
           "potential_ms_all": pot_ms,
           "solve_only": {"batched_ms": ms_batch_solve, "one_at_a_time_ms": ms_single_solve,
                          "speedup": ms_single_solve / ms_batch_solve,
                          "what": "cpm_batch_solve + cpm_batch_neutralize against cpm_solve + "
                                  "cpm_neutralize per context, b given"}}
    batch.close()
    for c in ctxs:
        c.close()
    return out


def run_learned(args, rank, world, local_rank):
    """Learned-guess form: the 512-atom electrode with the 200-ion set random-walked in
    0.1 A steps; the guess network is trained on `--train-frames` solver-generated frames
    and compared with the previous-step guess (Eq. 26) on `--heldout-frames` frames, all
    to 1e-6 relative residual.  Held-out frames are solved as one multi-RHS batch."""
    import torch

    from paper_2111_06704_gb300 import cpm
    from paper_2111_06704_gb300.guess import LearnedGuess

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    T, H = args.train_frames, args.heldout_frames
    t_gen = time.perf_counter()
    work = wl.walk_frames(T + H + 1, step=0.1, seed=wl.seed_for(4, rank))
    el, io = work.electrode, work.electrolyte
    n, F = el.n, io.frames
    tt = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    ctx = cpm.Context(el.box)
    ctx.cpm_build_E(tt(el.xyz), tt(el.alpha))
    chi = tt(el.chi)
    b = torch.empty((F, n), dtype=torch.float64, device=dev)
    qs = torch.empty(F, dtype=torch.float64, device=dev)
    qb = torch.zeros((F, n), dtype=torch.float64, device=dev)
    for f0 in range(0, F, 1024):
        f1 = min(F, f0 + 1024)
        ctx.cpm_potential(tt(io.xyz[f0:f1]), tt(io.q[f0:f1]), chi, b[f0:f1], qs[f0:f1])
    for f0 in range(0, F, 512):
        f1 = min(F, f0 + 512)
        ctx.cpm_solve(b[f0:f1], qb[f0:f1], tol=1e-9, maxit=2000)
    gen_s = time.perf_counter() - t_gen

    g = LearnedGuess(ctx, seed=rank)
    t_train = time.perf_counter()
    feat = g.features(b[1:T + 1], b[0:T], chi).reshape(-1, 32)
    target = (qb[1:T + 1] - qb[0:T]).reshape(-1).to(torch.float32).contiguous()
    k = min(T, 500) * n
    g.set_normalisation(feat[:k], target[:k])
    losses = g.train(feat, target, epochs=args.epochs, batch=65536, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t_train
    del feat, target

    test = slice(T + 1, T + H + 1)
    bt = b[test].contiguous()
    prev = qb[T:T + H].contiguous()

    def solve_prev():
        q = prev.clone()
        _, it, _ = ctx.cpm_solve(bt, q, use_guess=True, tol=TOL, maxit=2000)
        ctx.cpm_neutralize(q, qs[test].contiguous())
        return it

    bp = b[T:T + H].contiguous()

    def solve_learned():
        q0 = g.guess_frames(bt, bp, chi, prev)
        _, it, _ = ctx.cpm_solve(bt, q0, use_guess=True, tol=TOL, maxit=2000)
        ctx.cpm_neutralize(q0, qs[test].contiguous())
        return it

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, it

    def guess_only():
        return g.guess_frames(bt, bp, chi, prev)

    for _ in range(max(1, args.warmup)):
        solve_prev()
        solve_learned()
        guess_only()
    with ClockSampler(local_rank) as clocks:
        s_prev, it_prev = timed(solve_prev)
        s_learn, it_learn = timed(solve_learned)
        s_guess, _ = timed(guess_only)
    # plain per-frame FP64 Jacobi PCG from the previous-step guess, same GPU
    base = cpm.Context(el.box, precision=cpm.CPM_PREC_FP64, precond=cpm.CPM_PRECOND_JACOBI)
    base.cpm_build_E(tt(el.xyz), tt(el.alpha))
    nb = min(H, args.baseline_frames)
    q1 = torch.empty((1, n), dtype=torch.float64, device=dev)
    it_base = []

    def base_frames():
        for f in range(nb):
            q1.copy_(prev[f:f + 1])
            _, it, _ = base.cpm_solve(bt[f:f + 1], q1, use_guess=True, tol=TOL, maxit=5000)
            base.cpm_neutralize(q1, qs[T + 1 + f:T + 2 + f])
            it_base.append(int(it[0]))

    s_base, _ = timed(base_frames)
    if rank != 0:
        return
    value = H / s_learn
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": 1, "warmup": args.warmup, "ms_per_step": 1e3 * s_learn,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x6+fp16x3+fp8 (f32-accurate); guess network bf16 weights, f32 accumulation",
        "data": "synthetic",
        "config": {"workload": f"learned-guess form: two-sheet graphene N={n}, 200 ions "
                               f"random-walked 0.1 A/frame, {T} training frames, {H} held-out "
                               f"frames solved as one batch", "tol": TOL, "epochs": args.epochs},
        "learned": {"mean_iters": float(np.mean(it_learn)), "max_iters": int(np.max(it_learn)),
                    "solves_per_s": H / s_learn, "guess_ms": 1e3 * s_guess},
        "previous_step": {"mean_iters": float(np.mean(it_prev)), "max_iters": int(np.max(it_prev)),
                          "solves_per_s": H / s_prev},
        "iteration_gain": float(np.mean(it_prev) - np.mean(it_learn)),
        "baseline_fp64_per_frame_prev_guess": {"solves_per_s": nb / s_base,
                                               "mean_iters": float(np.mean(it_base)),
                                               "frames_timed": nb},
        "speedup_vs_fp64_per_frame": (H / s_learn) / (nb / s_base),
        "train": {"seconds": train_s, "first_loss": float(losses[0]),
                  "last_loss": float(losses[-1]), "steps": len(losses)},
        "generate_seconds": gen_s,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


SCALE_G, SCALE_RC = 0.15, 24.0  # the scale point's Ewald split (E does not depend on g)
SCALE_WORKLOAD = ("scale point: six stacked graphene sheets 7 A apart with 5% pinholes, "
                  "N={n}, {ions} ions, {frames} random-walk frames per step (E built once)")


def run_scale_point(args, rank, world, local_rank):
    """The default workload: the scale point (six stacked 90 x 52-cell graphene sheets with
    seeded pinholes, 106,568 electrode atoms, 221.4 x 221.5 x 105 A, 20,000 ions), with its
    16-frame batch and the learned initial guess.

    E (with P and d) is built once, timed apart (e_build_s, and the tensor-core tail's
    method-FLOP roofline).  A step is one charge solve of each of 16 consecutive frames of
    a 0.1 A random walk of the ions, as Sec. 8(d) defines a charge solve on a built E:
    cpm_potential of the 16 frames, the learned initial guess from the previous frames'
    charges, one PCG-DC over the 16 right-hand sides to 1e-6 relative residual, and
    cpm_neutralize.  The network is trained first on solver-generated frames of the same
    walk.  Beside it: the plain per-frame FP64 Jacobi PCG on the same GPU (the metric's
    comparator) on E_n widened to FP64 (cpm_build_E_copy; an FP64 k-space build is out of
    reach at this size), one frame per call from the previous-step guess (vs_baseline) and
    from zero."""
    import torch

    from paper_2111_06704_gb300 import cpm
    from paper_2111_06704_gb300.guess import LearnedGuess

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    T = min(args.train_frames, 48)
    H = args.rhs if args.rhs > 1 else 16
    work = wl.scale_walk(T + H + 1, step=0.1, seed=wl.seed_for(5, rank))
    el, io = work.electrode, work.electrolyte
    n, F = el.n, io.frames
    tt = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    with torch.cuda.stream(stream):
        ctx = cpm.Context(el.box, stream=stream.cuda_stream, g_ewald=SCALE_G,
                          rcut_real=SCALE_RC)
        xyz, alpha, chi = tt(el.xyz), tt(el.alpha), tt(el.chi)
        # E, P, d: one build to allocate the workspaces, one timed
        ctx.cpm_build_E(xyz, alpha)
        e0, e1 = events()
        with ClockSampler(local_rank) as build_clocks:
            torch.cuda.synchronize()
            e0.record(stream)
            ctx.cpm_build_E(xyz, alpha)
            e1.record(stream)
            torch.cuda.synchronize()
        build_s = e0.elapsed_time(e1) / 1e3
        binfo = ctx.cpm_get_info()
        ctx.cpm_release_workspace()

        # solver-generated training frames and the held-out batch's previous-step state
        b = torch.empty((F, n), dtype=torch.float64, device=dev)
        qs = torch.empty(F, dtype=torch.float64, device=dev)
        qb = torch.zeros((F, n), dtype=torch.float64, device=dev)
        for f0 in range(0, F, 16):
            f1 = min(F, f0 + 16)
            ctx.cpm_potential(tt(io.xyz[f0:f1]), tt(io.q[f0:f1]), chi, b[f0:f1], qs[f0:f1])
        for f0 in range(0, F, 16):
            f1 = min(F, f0 + 16)
            ctx.cpm_solve(b[f0:f1], qb[f0:f1], tol=1e-9, maxit=5000)
        g = LearnedGuess(ctx, seed=rank)
        feat = g.features(b[1:T + 1], b[0:T], chi).reshape(-1, 32)
        target = (qb[1:T + 1] - qb[0:T]).reshape(-1).to(torch.float32).contiguous()
        k = min(feat.shape[0], 500 * 512)
        g.set_normalisation(feat[:k], target[:k])
        losses = g.train(feat, target, epochs=args.epochs, batch=65536, lr=2e-3)
        del feat, target
        test = slice(T + 1, T + H + 1)
        ion_xyz, ion_q = tt(io.xyz[test]), tt(io.q[test])
        b_prev = b[T:T + H].contiguous()      # the previous frames' potentials ...
        q_prev = qb[T:T + H].contiguous()     # ... and converged charges (MD state)
        bt = torch.empty((H, n), dtype=torch.float64, device=dev)
        qst = torch.empty(H, dtype=torch.float64, device=dev)
        phase = {"potential": 0.0, "guess": 0.0, "solve": 0.0, "neutralize": 0.0}
        iters = []
        last_max_iters = [0]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]

        def step(q_out=None, record=True):
            ev[0].record(stream)
            ctx.cpm_potential(ion_xyz, ion_q, chi, bt, qst)
            ev[1].record(stream)
            q0 = g.guess_frames(bt, b_prev, chi, q_prev)
            ev[2].record(stream)
            _, it, _ = ctx.cpm_solve(bt, q0, use_guess=True, tol=TOL, maxit=5000)
            last_max_iters[0] = int(np.max(it))
            ev[3].record(stream)
            ctx.cpm_neutralize(q0, qst)
            ev[4].record(stream)
            if record:
                torch.cuda.synchronize()
                for name, a, z in zip(phase, ev[:4], ev[1:]):
                    phase[name] += a.elapsed_time(z)
                iters.append(float(np.mean(it)))
            if q_out is not None:
                q_out.copy_(q0, non_blocking=True)
            return q0

        for _ in range(args.warmup):
            step(record=False)
        phase = dict.fromkeys(phase, 0.0)
        iters.clear()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        launches0 = ctx.cpm_get_info()["launches"]
        t0, t1 = events()
        with ClockSampler(local_rank) as clocks:
            torch.cuda.synchronize()
            t0.record(stream)
            for _ in range(args.steps):
                q_last = step()
            t1.record(stream)
            torch.cuda.synchronize()
        launches = ctx.cpm_get_info()["launches"] - launches0
        ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, world)
        sinfo = ctx.cpm_get_info()  # the last step's solve
        solve_parts = {"solve_ms": sinfo["t_solve_ms"], "matvec_ms": sinfo["t_solve_matvec_ms"],
                       "replacement_ms": sinfo["t_solve_replace_ms"],
                       "replacements": sinfo["solve_replacements"],
                       "dc_apply_ms": sinfo["t_solve_dc_ms"],
                       "max_iterations": last_max_iters[0]}
        pot_parts = {"ion_structure_factors_ms": sinfo["t_pot_sf_ms"],
                     "kspace_ms": sinfo["t_pot_kspace_ms"],
                     "real_space_and_finish_ms": sinfo["t_pot_real_ms"]}
        # the same frames from the previous-step charges alone (Eq. 26), for the guess's gain
        q0 = q_prev.clone()
        _, it_prev, _ = ctx.cpm_solve(bt, q0, use_guess=True, tol=TOL, maxit=5000)
        # the step's charges against a tight solve of the same frames (FP64 reductions,
        # float-stored E): the error the 1e-6 residual leaves
        q_ref = q_prev.clone()
        ctx.cpm_solve(bt, q_ref, use_guess=True, tol=1e-10, maxit=5000)
        ctx.cpm_neutralize(q_ref, qst)
        q_err = float(((q_last - q_ref).norm(dim=1) / q_ref.norm(dim=1)).max())
        # the PCG matvec alone, one and 16 right-hand sides (E streamed per pass)
        mv = {}
        for r in (1, H):
            p = q_prev[:r].contiguous()
            out = torch.empty_like(p)
            ts = []
            for _ in range(4):
                ctx.cpm_apply_E(p, out)
                ts.append(ctx.cpm_get_info()["t_matvec_ms"])
            mv[r] = statistics.median(ts[1:])

        # end to end through the public API: the step's inputs from pinned host memory in,
        # the charges out, every step
        e2e = None
        if not args.no_e2e:
            hx = torch.tensor(io.xyz[test]).pin_memory()
            hq = torch.tensor(io.q[test]).pin_memory()
            hprev = q_prev.cpu().pin_memory()
            hout = torch.empty((H, n), dtype=torch.float64).pin_memory()

            def step_host():
                ion_xyz.copy_(hx, non_blocking=True)
                ion_q.copy_(hq, non_blocking=True)
                q_prev.copy_(hprev, non_blocking=True)
                step(q_out=hout, record=False)
                torch.cuda.synchronize()

            step_host()
            reps = max(1, min(args.steps, 3))
            c0 = time.perf_counter()
            for _ in range(reps):
                step_host()
            e2e_s = max_over_ranks((time.perf_counter() - c0) / reps, world)
            h2d = hx.numel() * 8 + hq.numel() * 8 + hprev.numel() * 8
            e2e = {"value": world * H / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": hout.numel() * 8,
                   "what": "ion positions and charges and the previous charges copied in from "
                           "pinned host memory, the step, the charges copied out"}

        # the metric's comparator: plain per-frame FP64 Jacobi PCG on the same GPU
        base = cpm.Context(el.box, stream=stream.cuda_stream, g_ewald=SCALE_G,
                           rcut_real=SCALE_RC, precision=cpm.CPM_PREC_FP64,
                           precond=cpm.CPM_PRECOND_JACOBI)
        base.cpm_build_E_copy(ctx)
        b1 = torch.empty((1, n), dtype=torch.float64, device=dev)
        qs1 = torch.empty(1, dtype=torch.float64, device=dev)
        q1 = torch.empty((1, n), dtype=torch.float64, device=dev)
        base_it = {"prev": [], "zero": []}

        def base_frame(f, guess):
            ctx.cpm_potential(ion_xyz[f:f + 1], ion_q[f:f + 1], chi, b1, qs1)
            if guess:
                q1.copy_(q_prev[f:f + 1])
            else:
                q1.zero_()
            _, it, _ = base.cpm_solve(b1, q1, use_guess=guess, tol=TOL, maxit=20000)
            base.cpm_neutralize(q1, qs1)
            base_it["prev" if guess else "zero"].append(int(it[0]))

        nb = max(1, min(H, args.baseline_frames))
        b0, b1e = events()
        torch.cuda.synchronize()
        b0.record(stream)
        for f in range(nb):
            base_frame(f, True)
        b1e.record(stream)
        torch.cuda.synchronize()
        base_prev_ms = b0.elapsed_time(b1e) / nb
        b0.record(stream)
        base_frame(0, False)
        b1e.record(stream)
        torch.cuda.synchronize()
        base_zero_ms = b0.elapsed_time(b1e)
        base_mv = []
        for _ in range(3):
            base.cpm_apply_E(q_prev[:1].contiguous(), b1)
            base_mv.append(base.cpm_get_info()["t_matvec_ms"])
        base.close()
    if rank != 0:
        return
    peaks, src = measured_peaks()
    value = world * H * 1000.0 / ms
    base_value = 1000.0 / base_prev_ms
    e_bytes = n * ((n + 127) // 128 * 128) * 4
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    n6, n3, n1 = binfo["tc_blocks"]
    tail_cols = 64 * (n6 + n3 + n1)
    method_flops = 2.0 * (n * (n + 1) / 2) * tail_cols
    issued_flops = 2.0 * (n * (n + 1) / 2) * 64 * (6 * n6 + 3 * n3 + n1)
    tc_ms = binfo["t_tc_ms"]
    sustained = peaks.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"])
    burst = peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"])
    achieved = method_flops / (tc_ms * 1e-3) / 1e12
    # the step's dominant kernel: the streamed 16-column matvec of the PCG iterations
    stream_tb, stream_note = stream_traffic()
    mv_launch_ms = solve_parts["matvec_ms"] / max(1, solve_parts["max_iterations"])
    mv_bytes = 4.0 * n * n + H * n * 4.0 + H * n * 8.0
    mv_achieved = mv_bytes / (mv_launch_ms * 1e-3) / 1e9
    step_roof = {"bound": "hbm", "achieved": mv_achieved, "peak": hbm, "unit": "GB/s",
                 "frac": mv_achieved / hbm,
                 "traffic": (stream_tb * n * n) if stream_tb else None,
                 "kernel": "k_matvec_stream (16-column float matvec of the PCG iterations, E "
                           "streamed by TMA once per iteration)",
                 "timed_region": "the timed steps: CUDA events around each iteration's matvec "
                                 "launch on the solve stream (last step's solve)",
                 "work": "algorithmic bytes per launch: N^2 x 4 (E) + 16 N x 4 (float "
                         "directions) + 16 N x 8 (FP64 products)",
                 "ms_per_launch": mv_launch_ms, "bytes_per_launch": mv_bytes,
                 "peak_source": f"{src} hbm_gbs (of measured)",
                 "traffic_source": stream_note}
    tail_tb, tail_note = tail_traffic()
    nt_tiles = (n + 255) // 256
    roof = {"bound": "tensor", "achieved": achieved, "peak": sustained, "unit": "TFLOP/s",
            "frac": achieved / sustained,
            "traffic": (tail_tb * nt_tiles * (nt_tiles + 1) // 2 * (n6 + n3 + n1))
            if tail_tb else None,
            "traffic_source": tail_note,
            "kernel": "k_ek_strip (tcgen05 k-space tail of the E build, all k-windows)",
            "timed_region": "the timed cpm_build_E (CUDA events around each window's "
                            "tensor-core launches, on the build stream)",
            "work": "method FLOPs: N(N+1)/2 lower-triangle entries x 2 x the tail's "
                    f"{tail_cols} operand columns",
            "peak_source": f"{src} bf16_tflops_sustained (of measured)",
            "frac_of_burst": achieved / burst,
            "issued_tflops": issued_flops / (tc_ms * 1e-3) / 1e12,
            "k_blocks_6_3_1_products": [n6, n3, n1], "k_blocks_fp8": binfo["tc_blocks_fp8"],
            "tc_ms": tc_ms, "tc_loop_ms": binfo["t_tc_loop_ms"], "head_ms": binfo["t_head_ms"]}
    mv_gbs = {r: e_bytes / (t * 1e-3) / 1e9 for r, t in mv.items()}
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": value / (world * base_value),
        "dtype": "bf16x6+fp16x3+fp8 (f32-accurate E), f64 vectors; guess network bf16",
        "data": "synthetic",
        "config": {"workload": SCALE_WORKLOAD.format(n=n, ions=io.n_ion, frames=H),
                   "electrode_atoms": n, "ions": io.n_ion, "frames_per_step": H,
                   "tol": TOL, "g_ewald": SCALE_G, "rcut_real": SCALE_RC,
                   "kvectors": binfo["m"], "precond": "PCG-DC (g=0.083, r_cut=8)",
                   "initial_guess": f"learned (trained on {T} solver-generated frames)",
                   "l2": f"inputs larger than L2: E {e_bytes / 1e9:.1f} GB streamed per "
                         "PCG iteration"},
        "baseline": {"value": base_value, "unit": "solves/s",
                     "what": "plain FP64 PCG, same GPU: E_n widened to FP64 "
                             "(cpm_build_E_copy), Jacobi, one frame per call, previous-step "
                             "guess; cpm_potential + cpm_solve + cpm_neutralize",
                     "frames_timed": nb, "mean_iters": float(np.mean(base_it["prev"])),
                     "zero_guess_value": 1000.0 / base_zero_ms,
                     "zero_guess_iters": base_it["zero"][0],
                     "matvec_ms": statistics.median(base_mv)},
        "e_build_s": build_s,
        "build_ms": {"phases": binfo["t_phase_ms"], "kspace": binfo["t_kspace_ms"],
                     "head": binfo["t_head_ms"], "tensor_core": tc_ms,
                     "tail_loop": binfo["t_tc_loop_ms"], "precond": binfo["t_precond_ms"],
                     "d_solve": binfo["t_dsolve_ms"]},
        "build_clocks": build_clocks.summary(),
        "phase_ms_per_step": {k: v / args.steps for k, v in phase.items()},
        "solve_breakdown": solve_parts,
        "potential_breakdown": pot_parts,
        "step_matvec": {
            "kernel": "k_matvec_stream (the 16 columns' inner matvec, E streamed once per "
                      "iteration)",
            "ms_per_launch": solve_parts["matvec_ms"] / max(1, solve_parts["max_iterations"]),
            "gbs": e_bytes / (solve_parts["matvec_ms"] / max(1, solve_parts["max_iterations"])
                              * 1e-3) / 1e9,
            "note": "matvec_ms: the iterations' matvec launches (one per iteration for the "
                    "group of 16 columns), events around each"},
        "mean_iters": statistics.mean(iters),
        "previous_step_guess_iters": float(np.mean(it_prev)),
        "q_rel_err_vs_tight_solve": q_err,
        "roofline": roof,
        "step_roofline": step_roof,
        "matvec_roofline": {"bound": "hbm", "kernel": "k_matvec_f32 (PCG matvec, E streamed "
                            "once per pass of up to four columns)",
                            "achieved": mv_gbs[1], "peak": hbm, "unit": "GB/s",
                            "frac": mv_gbs[1] / hbm, "ms": mv[1],
                            "bytes_per_launch": e_bytes,
                            f"ms_{H}_rhs": mv[H], "peak_source": f"{src} hbm_gbs"},
        "train": {"frames": T, "first_loss": float(losses[0]), "last_loss": float(losses[-1])},
        "peaks": {"source": src},
        "clocks": clocks.summary(),
        "gpu_launches": launches,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        build_cpu, solve_cpu = oracle_small_cell()
        line["cpu_baseline"] = {
            "value": 1.0 / solve_cpu, "unit": "solves/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": "one whole charge solve of the 512-atom two-sheet cell with 200 ions "
                      "(b^sol by direct sums, bordered dense solve), timed as it stands; the "
                      f"oracle's E build of that cell took {build_cpu:.1f} s",
            "e_build_s": build_cpu}
        est, _, desc = oracle_scale_sample(el, io.xyz[T + 1], io.q[T + 1], SCALE_G, SCALE_RC)
        line["cpu_baseline_scale_estimate"] = {"value": 1.0 / est, "unit": "solves/s",
                                               "cores": os.cpu_count(), "kind": "oracle",
                                               "sample": desc}
    print(json.dumps(line), flush=True)


def run_scale_learned(args, rank, world, local_rank):
    """Scale point with the learned initial guess: the ~106,600-atom electrode, its 20,000
    ions random-walked in 0.1 A steps; the guess network is trained on `--train-frames`
    (at most 48) solver-generated frames and compared with the previous-step guess (Eq. 26)
    on `--rhs` (16 unless given) held-out frames solved as one multi-right-hand-side batch,
    all to 1e-6 relative residual.  Streamed build as in the scale workload."""
    import torch

    from paper_2111_06704_gb300 import cpm
    from paper_2111_06704_gb300.guess import LearnedGuess

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    T, H = min(args.train_frames, 48), (args.rhs if args.rhs > 1 else 16)
    t_gen = time.perf_counter()
    work = wl.scale_walk(T + H + 1, step=0.1, seed=wl.seed_for(5, rank))
    el, io = work.electrode, work.electrolyte
    n, F = el.n, io.frames
    tt = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    ctx = cpm.Context(el.box, g_ewald=0.15, rcut_real=24.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.cpm_build_E(tt(el.xyz), tt(el.alpha))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    chi = tt(el.chi)
    b = torch.empty((F, n), dtype=torch.float64, device=dev)
    qs = torch.empty(F, dtype=torch.float64, device=dev)
    qb = torch.zeros((F, n), dtype=torch.float64, device=dev)
    for f0 in range(0, F, 16):
        f1 = min(F, f0 + 16)
        ctx.cpm_potential(tt(io.xyz[f0:f1]), tt(io.q[f0:f1]), chi, b[f0:f1], qs[f0:f1])
    for f0 in range(0, T + 1, H):
        f1 = min(T + 1, f0 + H)
        ctx.cpm_solve(b[f0:f1], qb[f0:f1], tol=1e-9, maxit=5000)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t_gen

    g = LearnedGuess(ctx, seed=rank)
    t_train = time.perf_counter()
    feat = g.features(b[1:T + 1], b[0:T], chi).reshape(-1, 32)
    target = (qb[1:T + 1] - qb[0:T]).reshape(-1).to(torch.float32).contiguous()
    k = min(feat.shape[0], 500 * 512)
    g.set_normalisation(feat[:k], target[:k])
    losses = g.train(feat, target, epochs=args.epochs, batch=65536, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t_train
    del feat, target

    test = slice(T + 1, T + H + 1)
    bt = b[test].contiguous()
    bp = b[T:T + H].contiguous()
    qst = qs[test].contiguous()

    # previous-step charges: frame T's, then each held-out frame's own converged solution
    prev = torch.empty((H, n), dtype=torch.float64, device=dev)
    prev[0] = qb[T]
    ref = torch.zeros((H, n), dtype=torch.float64, device=dev)
    ctx.cpm_solve(bt, ref, tol=1e-9, maxit=5000)
    prev[1:] = ref[:-1]

    def solve_prev():
        q = prev.clone()
        _, it, _ = ctx.cpm_solve(bt, q, use_guess=True, tol=TOL, maxit=5000)
        ctx.cpm_neutralize(q, qst)
        return it

    def solve_learned():
        q0 = g.guess_frames(bt, bp, chi, prev)
        _, it, _ = ctx.cpm_solve(bt, q0, use_guess=True, tol=TOL, maxit=5000)
        ctx.cpm_neutralize(q0, qst)
        return it

    def timed(fn):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        it = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t1, it

    for _ in range(max(1, args.warmup)):
        solve_prev()
        solve_learned()
    with ClockSampler(local_rank) as clocks:
        s_prev, it_prev = timed(solve_prev)
        s_learn, it_learn = timed(solve_learned)
        s_guess, _ = timed(lambda: g.guess_frames(bt, bp, chi, prev))
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": world * H / s_learn, "unit": "solves/s", "n_gpus": world,
        "steps": 1, "warmup": args.warmup, "ms_per_step": 1e3 * s_learn,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x6+fp16x3+fp8 (f32-accurate); guess network bf16 weights, f32 accumulation",
        "data": "synthetic",
        "config": {"workload": f"scale point with the learned guess: N={n}, {io.n_ion} ions "
                               f"random-walked 0.1 A/frame, {T} training frames, {H} held-out "
                               f"frames solved as one batch (build once)",
                   "electrode_atoms": n, "ions": io.n_ion, "rhs": H, "tol": TOL,
                   "g_ewald": 0.15, "rcut_real": 24.0, "epochs": args.epochs},
        "e_build_s": build_s,
        "learned": {"mean_iters": float(np.mean(it_learn)), "max_iters": int(np.max(it_learn)),
                    "solves_per_s": H / s_learn, "guess_ms": 1e3 * s_guess},
        "previous_step": {"mean_iters": float(np.mean(it_prev)), "max_iters": int(np.max(it_prev)),
                          "solves_per_s": H / s_prev},
        "iteration_gain": float(np.mean(it_prev) - np.mean(it_learn)),
        "train": {"seconds": train_s, "samples": T * n, "first_loss": float(losses[0]),
                  "last_loss": float(losses[-1]), "steps": len(losses)},
        "generate_seconds": gen_s,
        "clocks": clocks.summary(),
    }
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
    if args.workload == "batch":
        run_batch(args, rank, world, local_rank)
    elif args.workload == "learned":
        run_learned(args, rank, world, local_rank)
    elif args.workload == "matvec":
        run_matvec(args, rank, world, local_rank)
    elif args.workload == "scale":
        run_scale(args, rank, world, local_rank)
    elif args.workload == "scale-learned":
        run_scale_learned(args, rank, world, local_rank)
    elif args.workload == "precision":
        run_ours(args, rank, world, local_rank)
    elif args.workload == "build":
        run_build(args, rank, world, local_rank)
    elif args.workload == "potential":
        run_potential(args, rank, world, local_rank)
    else:
        run_scale_point(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
