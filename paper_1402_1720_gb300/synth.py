"""Seeded synthetic proton-CT workloads (inputs only).

This module generates proton histories the way the paper's data sets are
described (Sec. 2.1-2.2): a gantry rotated about the vertical axis in fixed
angular steps, straight-line entry-to-exit paths with Gaussian lateral exit
displacement standing in for multiple Coulomb scattering, and a WEPL that is
the line integral of relative stopping power (RSP) along the path, optionally
with Gaussian noise.  The paper's own phantoms (NEO digital head, CIRS 715-HN)
and its simulator are not available, so ellipsoid unions with the paper's RSP
values stand in for them.

It holds none of the hull-detection method's arithmetic: no classification,
no quantisation, no voxel traversal, no counting and no decisions.  Both the
CUDA path and the CPU oracle consume its arrays.

Coordinate convention (the paper gives none; the rotation axis is vertical,
Sec. 2.2 and its Fig. 2 caption):  world frame in mm with the origin at the
centre of the reconstruction volume and z the rotation axis.  At gantry angle
phi the beam runs along b = (cos phi, sin phi, 0); the lateral tracker axis is
e_u = (-sin phi, cos phi, 0) and the vertical one e_v = (0, 0, 1).  The entry
point is -T b + u_in e_u + v_in e_v and the exit point +T b + u_out e_u +
v_out e_v, with T the tracker half-separation.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Iterator, List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 20140202


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Reconstruction grid: nx*ny*nz voxels of sx*sy*sz mm centred on the
    isocentre, trackers at -T and +T along the beam."""
    nx: int
    ny: int
    nz: int
    sx: float
    sy: float
    sz: float
    T: float

    @property
    def n_voxels(self) -> int:
        return self.nx * self.ny * self.nz


@dataclasses.dataclass(frozen=True)
class Ellipsoid:
    center: Tuple[float, float, float]
    semi: Tuple[float, float, float]
    rsp: float


@dataclasses.dataclass
class Histories:
    """Structure-of-arrays proton histories, all float32 and equal length."""
    angle_deg: np.ndarray
    u_in: np.ndarray
    v_in: np.ndarray
    u_out: np.ndarray
    v_out: np.ndarray
    wepl: np.ndarray

    FIELDS = ("angle_deg", "u_in", "v_in", "u_out", "v_out", "wepl")

    def __len__(self) -> int:
        return int(self.angle_deg.shape[0])

    def arrays(self) -> List[np.ndarray]:
        return [getattr(self, f) for f in self.FIELDS]

    def take(self, idx) -> "Histories":
        return Histories(*[np.ascontiguousarray(a[idx]) for a in self.arrays()])

    @staticmethod
    def concat(parts: Sequence["Histories"]) -> "Histories":
        return Histories(*[np.concatenate([getattr(p, f) for p in parts])
                           for f in Histories.FIELDS])


@dataclasses.dataclass
class Workload:
    name: str
    geometry: Geometry
    phantom: List[Ellipsoid]
    histories: Histories


# ---------------------------------------------------------------- phantoms
def ellipsoid_phantom_c1() -> List[Ellipsoid]:
    """Tiny phantom: one centred ellipsoid, semi-axes 25, 28, 8 mm, RSP 1.0."""
    return [Ellipsoid((0.0, 0.0, 0.0), (25.0, 28.0, 8.0), 1.0)]


def head_phantom(scale: float = 0.75) -> List[Ellipsoid]:
    """Head-like painter's union (later entries override earlier ones):
    skull RSP 1.7, brain RSP 1.04 (skull minus a 6 mm shell), two air sinuses.
    RSP values follow Sec. 2.1 (bone, brain) with the sinuses as air.  The
    stated outer semi-axes (96, 120, 40) mm do not fit a 200 mm field of view,
    so they are scaled by `scale` (default 0.75 -> 72, 90, 30 mm)."""
    ax, ay, az = 96.0 * scale, 120.0 * scale, 40.0 * scale
    shell = 6.0
    return [
        Ellipsoid((0.0, 0.0, 0.0), (ax, ay, az), 1.7),
        Ellipsoid((0.0, 0.0, 0.0), (ax - shell, ay - shell, az - shell), 1.04),
        Ellipsoid((18.0, 60.0, 8.0), (10.0, 8.0, 6.0), 0.0),
        Ellipsoid((-18.0, 60.0, 8.0), (10.0, 8.0, 6.0), 0.0),
    ]


def random_phantom(rng: np.random.Generator, geom: Geometry) -> List[Ellipsoid]:
    """1-4 random ellipsoids inside the volume, RSP ~ U(0, 1.8)."""
    hx, hy, hz = geom.nx * geom.sx / 2, geom.ny * geom.sy / 2, geom.nz * geom.sz / 2
    out = []
    for _ in range(int(rng.integers(1, 5))):
        semi = (float(rng.uniform(0.15, 0.45) * hx), float(rng.uniform(0.15, 0.45) * hy),
                float(rng.uniform(0.15, 0.45) * hz))
        c = (float(rng.uniform(-1, 1) * (hx - semi[0]) * 0.8),
             float(rng.uniform(-1, 1) * (hy - semi[1]) * 0.8),
             float(rng.uniform(-1, 1) * (hz - semi[2]) * 0.8))
        out.append(Ellipsoid(c, semi, float(rng.uniform(0.0, 1.8))))
    return out


# ------------------------------------------------------------- path physics
def _endpoints(angle_deg, u_in, v_in, u_out, v_out, T):
    """World entry/exit points (float64) of the straight path model."""
    phi = np.deg2rad(angle_deg.astype(np.float64))
    c, s = np.cos(phi), np.sin(phi)
    u0, v0 = u_in.astype(np.float64), v_in.astype(np.float64)
    u1, v1 = u_out.astype(np.float64), v_out.astype(np.float64)
    p0 = np.stack([-T * c - u0 * s, -T * s + u0 * c, v0], axis=1)
    p1 = np.stack([T * c - u1 * s, T * s + u1 * c, v1], axis=1)
    return p0, p1


def _ellipsoid_interval(p0, d, e: Ellipsoid):
    """Parameter interval [t0, t1] (clipped to [0, 1]) of p0 + t d inside e;
    empty intervals come back with t0 == t1."""
    c = np.asarray(e.center)
    a = np.asarray(e.semi)
    q0 = (p0 - c) / a
    qd = d / a
    A = np.einsum("ij,ij->i", qd, qd)
    B = 2.0 * np.einsum("ij,ij->i", q0, qd)
    C = np.einsum("ij,ij->i", q0, q0) - 1.0
    disc = B * B - 4 * A * C
    ok = (disc > 0) & (A > 0)
    sq = np.sqrt(np.where(ok, disc, 0.0))
    Asafe = np.where(A > 0, A, 1.0)
    t0 = np.where(ok, (-B - sq) / (2 * Asafe), 0.0)
    t1 = np.where(ok, (-B + sq) / (2 * Asafe), 0.0)
    t0 = np.clip(t0, 0.0, 1.0)
    t1 = np.clip(t1, 0.0, 1.0)
    t1 = np.maximum(t1, t0)
    return t0, t1


def water_equivalent_path_length(p0, p1, phantom: Sequence[Ellipsoid]) -> np.ndarray:
    """Line integral of RSP along the segment p0 -> p1 through the painter's
    union (the last ellipsoid that contains a point sets its RSP)."""
    d = p1 - p0
    length = np.linalg.norm(d, axis=1)
    ivs = [_ellipsoid_interval(p0, d, e) for e in phantom]
    pts = [np.zeros(len(p0)), np.ones(len(p0))]
    for t0, t1 in ivs:
        pts += [t0, t1]
    ts = np.sort(np.stack(pts, axis=1), axis=1)
    wepl = np.zeros(len(p0))
    for k in range(ts.shape[1] - 1):
        a, b = ts[:, k], ts[:, k + 1]
        mid = 0.5 * (a + b)
        rsp = np.zeros(len(p0))
        for (t0, t1), e in zip(ivs, phantom):
            inside = (mid > t0) & (mid < t1)
            rsp = np.where(inside, e.rsp, rsp)
        wepl += rsp * (b - a) * length
    return wepl


def object_rsp_at(points: np.ndarray, phantom: Sequence[Ellipsoid]) -> np.ndarray:
    """RSP of the phantom at world points (n, 3)."""
    rsp = np.zeros(len(points))
    for e in phantom:
        q = (points - np.asarray(e.center)) / np.asarray(e.semi)
        inside = np.einsum("ij,ij->i", q, q) < 1.0
        rsp = np.where(inside, e.rsp, rsp)
    return rsp


def voxel_centres(geom: Geometry) -> np.ndarray:
    """World coordinates (V, 3) of the voxel centres, x fastest."""
    xs = (np.arange(geom.nx) + 0.5 - geom.nx / 2) * geom.sx
    ys = (np.arange(geom.ny) + 0.5 - geom.ny / 2) * geom.sy
    zs = (np.arange(geom.nz) + 0.5 - geom.nz / 2) * geom.sz
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def object_mask(geom: Geometry, phantom: Sequence[Ellipsoid]) -> np.ndarray:
    """The true object as a uint8 voxel mask: voxels whose centre lies inside
    any ellipsoid of the phantom (air cavities inside the head count as
    object, as a hull should enclose them)."""
    pts = voxel_centres(geom)
    inside = np.zeros(len(pts), bool)
    for e in phantom:
        q = (pts - np.asarray(e.center)) / np.asarray(e.semi)
        inside |= np.einsum("ij,ij->i", q, q) < 1.0
    return inside.astype(np.uint8)


# ---------------------------------------------------------------- histories
def make_histories(rng: np.random.Generator, geom: Geometry, phantom, angles_deg,
                   per_angle: int, u_half: float, v_half: float,
                   exit_sigma: float, wepl_sigma_rel: float, wepl_sigma_abs: float,
                   noise_free: bool = False, chunk: int = 1 << 20) -> Histories:
    """Histories grouped by gantry angle (acquisition order), uniform entry
    positions on the tracker face, Gaussian exit displacement, WEPL = RSP
    line integral + N(0, rel*WEPL + abs)."""
    angles = np.repeat(np.asarray(angles_deg, dtype=np.float32), per_angle)
    n = angles.shape[0]
    u_in = rng.uniform(-u_half, u_half, n).astype(np.float32)
    v_in = rng.uniform(-v_half, v_half, n).astype(np.float32)
    du = rng.normal(0.0, exit_sigma, n)
    dv = rng.normal(0.0, exit_sigma, n)
    noise = rng.normal(0.0, 1.0, n)
    u_out = (u_in + du).astype(np.float32)
    v_out = (v_in + dv).astype(np.float32)
    wepl = np.empty(n, dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        p0, p1 = _endpoints(angles[s:e], u_in[s:e], v_in[s:e], u_out[s:e], v_out[s:e], geom.T)
        w = water_equivalent_path_length(p0, p1, phantom)
        if not noise_free:
            w = w + noise[s:e] * (wepl_sigma_rel * w + wepl_sigma_abs)
        wepl[s:e] = w.astype(np.float32)
    return Histories(angles, u_in, v_in, u_out, v_out, wepl)


def _half_diag(g: Geometry) -> float:
    return math.hypot(g.nx * g.sx / 2, g.ny * g.sy / 2)


# ------------------------------------------------------------------ configs
CONFIG_NAMES = {
    1: "tiny-ellipsoid-64x64x8",
    2: "head-200x200x32-9e6",
    3: "head-400x400x128-streamed-9.9e7",
    4: "batched-48-scans",
    5: "serving-poisson",
}


def geometry_for(cid: int) -> Geometry:
    if cid == 1:
        return Geometry(64, 64, 8, 1.0, 1.0, 2.5, 100.0)
    if cid == 2:
        return Geometry(200, 200, 32, 1.0, 1.0, 2.5, 155.0)
    if cid == 3:
        return Geometry(400, 400, 128, 0.5, 0.5, 1.25, 155.0)
    raise ValueError(cid)


def make_config(cid: int, seed: Optional[int] = None, noise_free: bool = False,
                fraction: float = 1.0) -> Workload:
    """Configs 1-3 as one workload.  `fraction` < 1 keeps that fraction of
    histories per angle (a bounded sample of the same workload)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + cid if seed is None else seed))
    g = geometry_for(cid)
    if cid == 1:
        ph = ellipsoid_phantom_c1()
        per = max(1, int(round(2000 * fraction)))
        h = make_histories(rng, g, ph, np.arange(0, 360, 4), per, 35.0, 10.0,
                           1.0, 0.0, 0.5, noise_free)
    elif cid == 2:
        ph = head_phantom()
        per = max(1, int(round(100_000 * fraction)))
        h = make_histories(rng, g, ph, np.arange(0, 360, 4), per, 141.5, 40.0,
                           2.0, 0.01, 0.3, noise_free)
    elif cid == 3:
        ph = head_phantom()
        per = max(1, int(round(550_000 * fraction)))
        h = make_histories(rng, g, ph, np.arange(0, 360, 2), per, 141.5, 80.0,
                           2.0, 0.01, 0.3, noise_free)
    else:
        raise ValueError("configs 4 and 5 are multi-scan; use make_batch_scans")
    return Workload(CONFIG_NAMES[cid], g, ph, h)


def config3_chunk(k: int, seed: Optional[int] = None, fraction: float = 1.0,
                  noise_free: bool = False) -> Histories:
    """Chunk k (gantry angle 2k degrees) of config 3; each chunk has its own
    seed, so chunks can be generated independently and in any order."""
    base = SEED_BASE + 3 if seed is None else seed
    per = max(1, int(round(550_000 * fraction)))
    ang = np.arange(0, 360, 2)[k]
    rng = np.random.Generator(np.random.PCG64([base, k]))
    return make_histories(rng, geometry_for(3), head_phantom(), [ang], per, 141.5, 80.0,
                          2.0, 0.01, 0.3, noise_free)


def iter_config_chunks(cid: int, seed: Optional[int] = None, fraction: float = 1.0,
                       noise_free: bool = False) -> Iterator[Histories]:
    """Config 3 as per-angle chunks (the streamed acquisition of Sec. 4)."""
    assert cid == 3
    for k in range(180):
        yield config3_chunk(k, seed, fraction, noise_free)


BATCH_GRIDS = ((64, 64, 16), (128, 128, 32), (256, 256, 64))


@dataclasses.dataclass
class ScanSpec:
    geometry: Geometry
    phantom: List[Ellipsoid]
    n_histories: int
    seed: int


def batch_scan_specs(n_scans: int = 48, seed: Optional[int] = None,
                     hist_lo: float = 2e5, hist_hi: float = 2e7,
                     fraction: float = 1.0) -> List[ScanSpec]:
    """Config 4/5 scan distribution: grids from BATCH_GRIDS at 1x1x2.5 mm,
    1-4 random ellipsoids, log-uniform history counts."""
    base = SEED_BASE + 4 if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(base))
    out = []
    for k in range(n_scans):
        nx, ny, nz = BATCH_GRIDS[int(rng.integers(0, len(BATCH_GRIDS)))]
        g0 = Geometry(nx, ny, nz, 1.0, 1.0, 2.5, 0.0)
        T = float(np.ceil(_half_diag(g0) + 10.0))
        g = dataclasses.replace(g0, T=T)
        ph = random_phantom(rng, g)
        n = int(round(math.exp(rng.uniform(math.log(hist_lo), math.log(hist_hi))) * fraction))
        out.append(ScanSpec(g, ph, max(90, n), base * 1000 + k))
    return out


def scan_histories(spec: ScanSpec, angle_range: Optional[Tuple[int, int]] = None) -> Histories:
    """Histories of one batched/served scan: 90 angles at 4 deg, c2 noise.
    `angle_range` = (first, last+1) angle indices to generate only a part."""
    g = spec.geometry
    per = max(1, spec.n_histories // 90)
    a0, a1 = angle_range if angle_range is not None else (0, 90)
    parts = []
    for k in range(a0, a1):
        rng = np.random.Generator(np.random.PCG64([spec.seed, k]))
        parts.append(make_histories(rng, g, spec.phantom, [4.0 * k], per,
                                    _half_diag(g) + 1.0, g.nz * g.sz / 2,
                                    2.0, 0.01, 0.3))
    return Histories.concat(parts)


def batch_scan_part(job: Tuple) -> Histories:
    """Angles [a0, a1) of scan k of the 48-scan mix (`job` = (k, a0, a1) or
    (k, a0, a1, fraction)): concatenating the parts of consecutive angle
    ranges gives scan_histories(batch_scan_specs(48, fraction=fraction)[k]),
    so a scan can be generated in pieces by several processes."""
    k, a0, a1 = job[:3]
    fraction = job[3] if len(job) > 3 else 1.0
    return scan_histories(batch_scan_specs(48, fraction=fraction)[k], angle_range=(a0, a1))


def batch_scans_parallel(pool, fraction: float = 1.0, step: int = 10) -> List[Histories]:
    """All 48 scans of the mix, generated by `pool` (a multiprocessing pool)
    in pieces of `step` angles; identical to scan_histories of each spec."""
    jobs = [(k, a, min(90, a + step), fraction) for k in range(48) for a in range(0, 90, step)]
    parts = pool.map(batch_scan_part, jobs)
    return [Histories.concat([p for j, p in zip(jobs, parts) if j[0] == k]) for k in range(48)]


def tiny_random_case(rng: np.random.Generator, n: int, geom: Geometry,
                     span: float = 1.3) -> Histories:
    """Random histories for small parity fuzzing: random angles, positions
    spread over `span` times the volume, WEPL drawn so that roughly a third
    miss (< 1), a third hit (> 5) and the rest fall between."""
    hd = _half_diag(geom) * span
    hz = geom.nz * geom.sz / 2 * span
    angle = rng.uniform(-720.0, 720.0, n).astype(np.float32)
    u_in = rng.uniform(-hd, hd, n).astype(np.float32)
    v_in = rng.uniform(-hz, hz, n).astype(np.float32)
    u_out = (u_in + rng.normal(0, 0.3 * hd, n)).astype(np.float32)
    v_out = (v_in + rng.normal(0, 0.3 * hz, n)).astype(np.float32)
    wepl = rng.choice(np.array([0.5, 3.0, 7.0], dtype=np.float32), n)
    return Histories(angle, u_in, v_in, u_out, v_out, wepl)
