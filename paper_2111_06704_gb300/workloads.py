"""Seeded synthetic workloads for the SR-CPM electrode-charge path.

This module only places atoms and ions: it holds none of the method's arithmetic
(no Ewald sums, no solves).  Both the CUDA path and the CPU oracle take its arrays as
inputs, so the two share inputs and nothing else.

Geometry (the paper's graphene electrochemical cell, Sec. IV A, Fig. 4, restated for
the workloads used here):

* Graphene sheets are built from rectangular 4-atom cells of ``a x b`` (2.46 x 4.26 A)
  with fractional basis x in {0, 0, 1/2, 1/2}, y in {0, 1/3, 1/2, 5/6}.  Two sheets sit at
  z = 0 and z = 30 A in a box padded 3x along z (Lz = 90 A).
* Ions are +1/-1 point charges placed uniformly at random in the slit 3 < z < 27 A,
  optionally with a minimum separation (minimum image in x, y; plain distance in z).
* Every generator draws from ``numpy.random.default_rng(seed)`` with
  ``seed = 20211106 + 1000 * config_id + frame_batch`` unless a seed is passed.

Units: Angstrom, elementary charge, volt.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 20211106

# Rectangular graphene cell as given for the workloads (2.46 x 4.26 A).
CELL_A = 2.46
CELL_B = 4.26
BASIS_FRAC = np.array([[0.0, 0.0], [0.0, 1.0 / 3.0], [0.5, 0.5], [0.5, 5.0 / 6.0]])


def seed_for(config_id: int, frame_batch: int = 0) -> int:
    return SEED_BASE + 1000 * config_id + frame_batch


@dataclasses.dataclass
class Electrode:
    """Electrode atoms: xyz[N,3] (A), alpha[N] (1/A), chi[N] (V)."""

    xyz: np.ndarray
    alpha: np.ndarray
    chi: np.ndarray
    box: tuple  # (Lx, Ly, Lz)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


@dataclasses.dataclass
class Electrolyte:
    """Point-charge ions: xyz[F, Nion, 3] (A) and q[F, Nion] (e)."""

    xyz: np.ndarray
    q: np.ndarray

    @property
    def frames(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_ion(self) -> int:
        return int(self.xyz.shape[1])


def graphene_sheet(nx: int, ny: int, z: float, a: float = CELL_A, b: float = CELL_B) -> np.ndarray:
    """One flat sheet of nx*ny rectangular 4-atom cells at height z; returns [4*nx*ny, 3]."""
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel()], axis=1).astype(np.float64)
    pts = (cells[:, None, :] + BASIS_FRAC[None, :, :]).reshape(-1, 2)
    out = np.empty((pts.shape[0], 3))
    out[:, 0] = pts[:, 0] * a
    out[:, 1] = pts[:, 1] * b
    out[:, 2] = z
    return out


def ideal_graphene_cell(bond: float = 1.0):
    """Rectangular 4-atom cell of the ideal honeycomb with the given bond length.

    Returns (a, b): a = sqrt(3) * bond, b = 3 * bond, for use with ``graphene_sheet``."""
    return math.sqrt(3.0) * bond, 3.0 * bond


def two_sheet_electrode(nx: int, ny: int, gap: float = 30.0, lz_pad: float = 3.0,
                        alpha: float = 1.979, chi_low: float = -0.5, chi_high: float = 0.5,
                        a: float = CELL_A, b: float = CELL_B) -> Electrode:
    """Two sheets at z = 0 and z = gap in an (nx*a, ny*b, lz_pad*gap) box."""
    low = graphene_sheet(nx, ny, 0.0, a, b)
    high = graphene_sheet(nx, ny, gap, a, b)
    xyz = np.concatenate([low, high], axis=0)
    n_half = low.shape[0]
    chi = np.concatenate([np.full(n_half, chi_low), np.full(n_half, chi_high)])
    alpha_arr = np.full(xyz.shape[0], alpha, dtype=np.float64)
    box = (nx * a, ny * b, lz_pad * gap)
    return Electrode(xyz=xyz, alpha=alpha_arr, chi=chi, box=box)


def _min_image_dist2(p: np.ndarray, pts: np.ndarray, lx: float, ly: float) -> np.ndarray:
    d = pts - p
    d[:, 0] -= lx * np.round(d[:, 0] / lx)
    d[:, 1] -= ly * np.round(d[:, 1] / ly)
    return np.einsum("ij,ij->i", d, d)


def random_ions(rng: np.random.Generator, n_cat: int, n_an: int, box, zlo: float = 3.0,
                zhi: float = 27.0, min_sep: float | None = 2.5, max_tries: int = 2_000_000):
    """Uniform ions in zlo < z < zhi by rejection sampling with an optional minimum
    separation (minimum image in x and y, plain distance in z).  Cations first."""
    lx, ly, _ = box
    n = n_cat + n_an
    pts = np.empty((n, 3))
    placed = 0
    tries = 0
    sep2 = None if min_sep is None else min_sep * min_sep
    while placed < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("ion placement did not finish; lower the density or min_sep")
        p = np.array([rng.uniform(0.0, lx), rng.uniform(0.0, ly), rng.uniform(zlo, zhi)])
        if sep2 is not None and placed > 0:
            if np.min(_min_image_dist2(p, pts[:placed], lx, ly)) < sep2:
                continue
        pts[placed] = p
        placed += 1
    q = np.concatenate([np.ones(n_cat), -np.ones(n_an)])
    return pts, q


def perturb_frames(rng: np.random.Generator, base_xyz: np.ndarray, frames: int, sigma: float,
                   box, zlo: float = 3.0, zhi: float = 27.0) -> np.ndarray:
    """Frames of Gaussian-perturbed copies of base_xyz; x, y wrap, z reflects into (zlo, zhi)."""
    lx, ly, _ = box
    out = base_xyz[None, :, :] + rng.normal(0.0, sigma, size=(frames,) + base_xyz.shape)
    out[..., 0] %= lx
    out[..., 1] %= ly
    out[..., 2] = _reflect(out[..., 2], zlo, zhi)
    return out


def random_walk_frames(rng: np.random.Generator, start_xyz: np.ndarray, frames: int, step: float,
                       box, zlo: float = 3.0, zhi: float = 27.0) -> np.ndarray:
    """Consecutive frames of an isotropic Gaussian random walk with reflecting z walls."""
    lx, ly, _ = box
    out = np.empty((frames,) + start_xyz.shape)
    cur = start_xyz.copy()
    for f in range(frames):
        cur = cur + rng.normal(0.0, step, size=cur.shape)
        cur[:, 0] %= lx
        cur[:, 1] %= ly
        cur[:, 2] = _reflect(cur[:, 2], zlo, zhi)
        out[f] = cur
    return out


def _reflect(z: np.ndarray, lo: float, hi: float) -> np.ndarray:
    span = hi - lo
    t = np.mod(z - lo, 2.0 * span)
    return lo + np.where(t > span, 2.0 * span - t, t)


# ----------------------------------------------------------------------------------------
# The workloads.
# ----------------------------------------------------------------------------------------

# Physical parameters shared by the two-sheet workloads.
G_EWALD = 0.3       # Ewald splitting parameter (1/A)
RCUT_REAL = 12.0    # real-space cutoff (A)
KSPACE_EPS = 1e-8   # k-space truncation: exp(-Kc^2 / 4g^2) = eps
ALPHA = 1.979       # Gaussian inverse width of the electrode charges (1/A)
G_DC = 0.083        # PCG-DC screening factor (1/A), Sec. IV A
RCUT_DC = 8.0       # PCG-DC neighbour cutoff (A)


@dataclasses.dataclass
class Workload:
    name: str
    electrode: Electrode
    electrolyte: Electrolyte


def small_cell(seed: int | None = None) -> Workload:
    """512 electrode atoms (two 8x8-cell sheets), 100 cations + 100 anions, one frame."""
    el = two_sheet_electrode(8, 8)
    rng = np.random.default_rng(seed_for(1) if seed is None else seed)
    ions, q = random_ions(rng, 100, 100, el.box, min_sep=2.5)
    return Workload("two-sheet graphene N=512, 200 ions", el,
                    Electrolyte(ions[None], q[None]))


def precision_cell(seed: int | None = None, cells: int = 40, n_ion: int = 2000) -> Workload:
    """12,800 electrode atoms (two 40x40-cell sheets), 1,000 + 1,000 ions, one frame."""
    el = two_sheet_electrode(cells, cells)
    rng = np.random.default_rng(seed_for(2) if seed is None else seed)
    ions, q = random_ions(rng, n_ion // 2, n_ion // 2, el.box, min_sep=2.5)
    return Workload(f"two-sheet graphene N={el.n}, {n_ion} ions", el,
                    Electrolyte(ions[None], q[None]))


def frame_batch(frames: int = 256, n_ion: int = 2000, sigma: float = 0.5,
                seed: int | None = None) -> Workload:
    """The 512-atom electrode with `frames` Gaussian-perturbed (sigma) 2,000-ion frames.

    2,000 ions do not fit the 19.68 x 34.08 x 24 A slit with a 2.5 A separation, so the
    base frame is drawn without one (electrode-ion distances stay >= 3 A)."""
    el = two_sheet_electrode(8, 8)
    rng = np.random.default_rng(seed_for(3) if seed is None else seed)
    base, q = random_ions(rng, n_ion // 2, n_ion // 2, el.box, min_sep=None)
    xyz = perturb_frames(rng, base, frames, sigma, el.box)
    return Workload(f"two-sheet graphene N=512, {frames} frames x {n_ion} ions", el,
                    Electrolyte(xyz, np.broadcast_to(q, (frames, n_ion)).copy()))


def walk_frames(frames: int, step: float = 0.1, seed: int | None = None,
                start: Electrolyte | None = None) -> Workload:
    """The 512-atom electrode with ions (default: the 200-ion small-cell set) random-walked
    with isotropic Gaussian steps, one frame per step."""
    base = small_cell() if start is None else None
    el = two_sheet_electrode(8, 8)
    ions0 = base.electrolyte.xyz[0] if start is None else start.xyz[0]
    q = base.electrolyte.q[0] if start is None else start.q[0]
    rng = np.random.default_rng(seed_for(4) if seed is None else seed)
    xyz = random_walk_frames(rng, ions0, frames, step, el.box)
    return Workload(f"two-sheet graphene N=512, {frames} random-walk frames", el,
                    Electrolyte(xyz, np.broadcast_to(q, (frames, q.shape[0])).copy()))


def ragged_systems(count: int = 32, n_lo: int = 500, n_hi: int = 8000, seed: int | None = None):
    """`count` independent two-sheet systems with electrode counts drawn uniformly in
    [n_lo, n_hi]; each sheet is near-square with 8*nx*ny ~ N; ions = round(N*200/512),
    rounded to an even count."""
    rng = np.random.default_rng(seed_for(3, 1) if seed is None else seed)
    out = []
    for _ in range(count):
        target = int(rng.integers(n_lo, n_hi + 1))
        cells = max(1, round(target / 8))
        # near-square sheet in length: nx*a ~ ny*b
        nx = max(1, round(math.sqrt(cells * CELL_B / CELL_A)))
        ny = max(1, round(cells / nx))
        el = two_sheet_electrode(nx, ny)
        n_ion = 2 * max(1, round(el.n * 200 / 512 / 2))
        ions, q = random_ions(rng, n_ion // 2, n_ion // 2, el.box, min_sep=None)
        out.append(Workload(f"two-sheet graphene N={el.n}, {n_ion} ions", el,
                            Electrolyte(ions[None], q[None])))
    return out


def stacked_electrode(rng: np.random.Generator, nx: int = 90, ny: int = 52, sheets: int = 6,
                      spacing: float = 7.0, lz: float = 105.0, hole_frac: float = 0.05,
                      r_lo: float = 3.0, r_hi: float = 8.0, alpha: float = 1.979,
                      chi: float = 0.5) -> Electrode:
    """`sheets` graphene sheets of nx x ny cells, `spacing` apart from z = 0, each with
    seeded circular pinholes (radius uniform in [r_lo, r_hi], minimum image in x, y) cut
    until at least `hole_frac` of its atoms are removed; sheet potentials alternate
    -chi, +chi."""
    lx, ly = nx * CELL_A, ny * CELL_B
    parts, chis = [], []
    for s in range(sheets):
        pts = graphene_sheet(nx, ny, s * spacing)
        keep = np.ones(pts.shape[0], dtype=bool)
        while np.count_nonzero(~keep) < hole_frac * pts.shape[0]:
            c = np.array([rng.uniform(0.0, lx), rng.uniform(0.0, ly), s * spacing])
            r = rng.uniform(r_lo, r_hi)
            keep &= _min_image_dist2(c, pts, lx, ly) >= r * r
        parts.append(pts[keep])
        chis.append(np.full(int(keep.sum()), chi if s % 2 else -chi))
    xyz = np.concatenate(parts, axis=0)
    return Electrode(xyz=xyz, alpha=np.full(xyz.shape[0], alpha), chi=np.concatenate(chis),
                     box=(lx, ly, lz))


def scale_point(seed: int | None = None, n_ion: int = 20000, rhs: int = 1) -> Workload:
    """Six stacked 90 x 52-cell sheets 7 A apart with 5% pinholes (~106,700 atoms) in a
    221.4 x 221.52 x 105 A box; n_ion ions (half +1, half -1) spread evenly over the five
    gaps, each at least 2 A from both sheets and 2.5 A from the other ions of its gap;
    `rhs` frames, Gaussian perturbations (0.5 A) of the first, z reflected into the band."""
    rng = np.random.default_rng(seed_for(5) if seed is None else seed)
    el = stacked_electrode(rng)
    gaps = 5
    per = n_ion // gaps
    xyz, q = [], []
    for g_ in range(gaps):
        zlo, zhi = 7.0 * g_ + 2.0, 7.0 * (g_ + 1) - 2.0
        pts, qq = random_ions(rng, per // 2, per - per // 2, el.box, zlo=zlo, zhi=zhi,
                              min_sep=2.5)
        xyz.append(pts)
        q.append(qq)
    base = np.concatenate(xyz, axis=0)
    qv = np.concatenate(q)
    frames = [base]
    for _ in range(rhs - 1):
        f = base + rng.normal(0.0, 0.5, size=base.shape)
        f[:, 0] %= el.box[0]
        f[:, 1] %= el.box[1]
        for g_ in range(gaps):  # reflect each ion back into its own band
            sel = (base[:, 2] >= 7.0 * g_) & (base[:, 2] < 7.0 * (g_ + 1))
            f[sel, 2] = _reflect(f[sel, 2], 7.0 * g_ + 2.0, 7.0 * (g_ + 1) - 2.0)
        frames.append(f)
    return Workload(f"six stacked graphene sheets with pinholes N={el.n}, {len(qv)} ions",
                    el, Electrolyte(np.stack(frames), np.broadcast_to(qv, (rhs, len(qv))).copy()))


def scale_walk(frames: int, step: float = 0.1, seed: int | None = None) -> Workload:
    """The scale-point electrode and ions (frame 0 of scale_point) random-walked with
    isotropic Gaussian steps, one frame per step, each ion reflected back into its own gap
    (at least 2 A from both sheets); x and y wrap."""
    base = scale_point(seed=seed, rhs=1)
    el, ions0, q = base.electrode, base.electrolyte.xyz[0], base.electrolyte.q[0]
    rng = np.random.default_rng((seed_for(5) if seed is None else seed) + 1)
    gap = np.floor(ions0[:, 2] / 7.0).astype(int)
    out = np.empty((frames,) + ions0.shape)
    cur = ions0.copy()
    for f in range(frames):
        cur = cur + rng.normal(0.0, step, size=cur.shape)
        cur[:, 0] %= el.box[0]
        cur[:, 1] %= el.box[1]
        cur[:, 2] = _reflect(cur[:, 2], 7.0 * gap + 2.0, 7.0 * (gap + 1) - 2.0)
        out[f] = cur
    return Workload(f"{base.name}, {frames} random-walk frames", el,
                    Electrolyte(out, np.broadcast_to(q, (frames, q.shape[0])).copy()))
