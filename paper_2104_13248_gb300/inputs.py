"""Seeded synthetic inputs: workload presets, random numbers and phantom draws.

This module holds no arithmetic of the reconstruction method (no projection
matrices, sampling, filtering or back-projection). It only produces numbers:
the geometry presets of the five workloads, SplitMix64 random streams, and
ellipsoid phantom parameters. Both the CUDA path and the FP64 CPU oracle
consume what it returns; neither is imported here.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then the output mix
z = (z ^ z>>30) * 0xBF58476D1CE4E5B9; z = (z ^ z>>27) * 0x94D049BB133111EB;
z ^ z>>31. Uniform doubles take the top 53 bits.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def _mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


class SplitMix64:
    """Sequential SplitMix64 stream."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + _GAMMA) & _M64
        return _mix(self.state)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def gauss(self) -> float:
        # Box-Muller on two uniforms in (0, 1].
        u1 = 1.0 - self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def uniform_array(seed: int, shape, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Counter-based SplitMix64: element n is mix(seed + (n+1)*gamma), float64."""
    n = int(np.prod(shape))
    out = np.empty(n, dtype=np.float64)
    chunk = 1 << 22
    with np.errstate(over="ignore"):
        for b in range(0, n, chunk):
            e = min(n, b + chunk)
            z = (np.uint64(seed & _M64)
                 + (np.arange(b + 1, e + 1, dtype=np.uint64) * np.uint64(_GAMMA)))
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
            out[b:e] = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (lo + (hi - lo) * out).reshape(shape)


# ---------------------------------------------------------------------------
# Workload presets (sizes from the five workloads this library is built for)
# ---------------------------------------------------------------------------

def _geom(np_, nu, nv, du, dv, n, s, sid=1000.0, sdd=1500.0):
    return dict(sid=sid, sdd=sdd, np=np_, angles=None, nu=nu, nv=nv, du=du, dv=dv,
                u_off=0.0, v_off=0.0, nx=n, ny=n, nz=n, sx=s, sy=s, sz=s,
                ox=0.0, oy=0.0, oz=0.0)


PRESETS = {
    # FDK at CPU-oracle size: 90 views, 128^2 @ 0.8 mm -> 64^3 @ 1 mm.
    "c1_small": dict(geom=_geom(90, 128, 128, 0.8, 0.8, 64, 1.0), n_ell=10,
                     axes=(5.0, 25.0), seed=1),
    # FDK: 360 views, 512^2 @ 0.4 mm -> 256^3 @ 0.5 mm.
    "c2_fdk256": dict(geom=_geom(360, 512, 512, 0.4, 0.4, 256, 0.5), n_ell=30,
                      axes=(3.0, 40.0), seed=2),
    # Paper scale: 496 views, 1248x960 @ 0.3 mm -> 512^3 @ 0.25 mm.
    "c3_paper": dict(geom=_geom(496, 1248, 960, 0.3, 0.3, 512, 0.25), n_ell=50,
                     axes=(2.0, 50.0), seed=3),
    # Differentiable LS: 180 views, 512^2 @ 0.4 mm -> 4 x 256^3 @ 0.5 mm.
    "c4_diff": dict(geom=_geom(180, 512, 512, 0.4, 0.4, 256, 0.5), n_ell=30,
                    axes=(3.0, 40.0), seed=100, batch=4, iters=20),
    # Learned few-view: 60 of 360 views, 512^2 @ 0.4 mm -> 256^3 @ 0.5 mm.
    "c5_learned": dict(geom=_geom(360, 512, 512, 0.4, 0.4, 256, 0.5), n_ell=30,
                       axes=(3.0, 40.0), seed=1000, few=60, train_pairs=256,
                       crop=128, heldout_seed=5000, heldout=32),
}


# The paper's problem grid (Section 4, table of problem sizes): square
# detectors of 256, 512 or 1024 pixels, 512 views over 360 deg, volumes of
# 256^3, 512^3, 1024^3 and 1300^3. The paper gives no geometry for them; these
# keep the source distances of the workloads above, a 204.8 mm detector and a
# 128 mm volume (the footprint of the 512^2 / 256^3 workload).
PROBLEMS = {
    "P1": (256, 256), "P2": (256, 512), "P3": (256, 1024),
    "P4": (512, 256), "P5": (512, 512), "P6": (512, 1024),
    "P7": (1024, 256), "P8": (1024, 512), "P9": (1024, 1024),
    "P10": (1024, 1300),
}


def paper_problem(label: str, views: int = 512) -> dict:
    """Geometry of problem ``label`` (detector n x n, volume m^3, 512 views)."""
    n, m = PROBLEMS[label]
    return _geom(views, n, n, 204.8 / n, 204.8 / n, m, 128.0 / m)


def preset(name: str) -> dict:
    p = PRESETS[name]
    out = dict(p)
    out["geom"] = dict(p["geom"])
    return out


def scaled_geom(g: dict, **kw) -> dict:
    """Copy of a geometry dict with some fields replaced."""
    out = dict(g)
    out.update(kw)
    return out


# ---------------------------------------------------------------------------
# Ellipsoid phantoms
# ---------------------------------------------------------------------------

def _quat_to_rot(q):
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def fov_limits(g: dict) -> tuple[float, float]:
    """Radius and half-height (mm) of the region every ellipsoid must fit in.

    Radius: the largest centred cylinder seen by every view (half fan angle
    atan(nu*du/2 / sdd) at distance sid), capped by the volume's half-width.
    Half-height: the volume's half-height, capped by the detector's
    half-height scaled back to the far edge of that cylinder.
    """
    half_u = 0.5 * g["nu"] * g["du"]
    half_v = 0.5 * g["nv"] * g["dv"]
    r_fan = g["sid"] * math.sin(math.atan(half_u / g["sdd"]))
    r_vol = 0.5 * min(g["nx"] * g["sx"], g["ny"] * g["sy"])
    r = min(r_fan, r_vol)
    h_vol = 0.5 * g["nz"] * g["sz"]
    h_det = half_v * (g["sid"] - r) / g["sdd"]
    return r, min(h_vol, h_det)


def random_ellipsoids(seed: int, n: int, axes: tuple[float, float], g: dict,
                      rho: tuple[float, float] = (0.0, 1.0)) -> np.ndarray:
    """n ellipsoids as [n][16] rows: cx, cy, cz, ax, ay, az, R (3x3 row-major,
    body -> world), rho.

    Semi-axes U[axes], density U[rho], rotation from a normalised Gaussian
    quaternion (uniform on SO(3)). The centre is drawn uniformly in the
    cylinder where the ellipsoid's bounding sphere stays inside 0.9 x the
    field of view (``fov_limits``); the semi-axes are redrawn when no such
    centre exists. Overlapping ellipsoids add.
    """
    rng = SplitMix64(seed)
    R_fov, H = fov_limits(g)
    out = np.zeros((n, 16), dtype=np.float64)
    for e in range(n):
        for _ in range(10000):
            a = [rng.uniform(*axes) for _ in range(3)]
            rmax = 0.9 * R_fov - max(a)
            zmax = 0.9 * H - max(a)
            if rmax >= 0.0 and zmax >= 0.0:
                break
        else:
            raise ValueError("semi-axes too large for the field of view")
        rad = rmax * math.sqrt(rng.uniform())
        phi = 2.0 * math.pi * rng.uniform()
        cz = rng.uniform(-zmax, zmax)
        q = np.array([rng.gauss() for _ in range(4)])
        q /= np.linalg.norm(q)
        R = _quat_to_rot(q)
        out[e, 0:3] = (rad * math.cos(phi), rad * math.sin(phi), cz)
        out[e, 3:6] = a
        out[e, 6:15] = R.reshape(-1)
        out[e, 15] = rng.uniform(*rho)
    return out


def sphere(radius: float, rho: float = 1.0, centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """One sphere in the [1][16] ellipsoid row format."""
    out = np.zeros((1, 16), dtype=np.float64)
    out[0, 0:3] = centre
    out[0, 3:6] = radius
    out[0, 6:15] = np.eye(3).reshape(-1)
    out[0, 15] = rho
    return out


def density_at(ellipsoids: np.ndarray, x, y, z) -> np.ndarray:
    """Phantom density at world points (broadcast arrays of mm coordinates)."""
    x, y, z = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float), np.asarray(z, float))
    d = np.zeros(x.shape, dtype=np.float64)
    for E in np.asarray(ellipsoids).reshape(-1, 16):
        R = E[6:15].reshape(3, 3)
        p = np.stack([x - E[0], y - E[1], z - E[2]], axis=-1)
        b = p @ R  # R^T p, row-vector form
        r2 = (b[..., 0] / E[3]) ** 2 + (b[..., 1] / E[4]) ** 2 + (b[..., 2] / E[5]) ** 2
        d += np.where(r2 <= 1.0, E[15], 0.0)
    return d


def surface_distance_mask(ellipsoids: np.ndarray, x, y, z, margin: float) -> np.ndarray:
    """True where a point is at least ``margin`` mm (approximately: scaled
    along the normalised radius) away from every ellipsoid surface."""
    x, y, z = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float), np.asarray(z, float))
    ok = np.ones(x.shape, dtype=bool)
    for E in np.asarray(ellipsoids).reshape(-1, 16):
        R = E[6:15].reshape(3, 3)
        p = np.stack([x - E[0], y - E[1], z - E[2]], axis=-1)
        b = p @ R
        amin = min(E[3], E[4], E[5])
        r = np.sqrt((b[..., 0] / E[3]) ** 2 + (b[..., 1] / E[4]) ** 2 + (b[..., 2] / E[5]) ** 2)
        # |r - 1| * min semi-axis under-estimates the true distance to the surface
        ok &= np.abs(r - 1.0) * amin >= margin
    return ok
