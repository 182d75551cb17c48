"""FP64 CPU oracle for cone-beam back-projection (ctypes wrapper of oracle.c).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. The product path
(``paper_2104_13248_gb300``) never imports it and shares no code with it.

Each function follows a passage of Chen et al., ICS '21:
  matrices          Section 2.1.1 (pinhole 3x4 matrix; explicit form is our reading)
  backproject       Listing 1 with the sampling of Listing 2, in double
  forward_project   the exact transpose of ``backproject`` (matched adjoint)
  ramp_filter       FDK pre-filtering assumed by Section 2.1.2 (our reading:
                    cosine weight + discrete Ram-Lak, linear convolution)
  fdk               ramp_filter then backproject with scale pi/np
  phantom_project   analytic line integrals of an ellipsoid phantom (input data)
  siddon            ray-driven line integrals through a voxel grid (checks the
                    phantom projector's geometry)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def compile_source(src: str, out: str) -> str:
    """gcc build of an oracle source file: FP64, OpenMP, no FMA contraction."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-std=c11", src, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (skipped when fresh)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    return compile_source(src, _SO)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_SO)
    return _lib


class _Bound:
    """Context manager that points every routine of this module at another
    build of oracle.c (used by the tests that plant mistakes in a copy of the
    source to show that the pins catch them)."""

    def __init__(self, so_path: str):
        self.lib = ctypes.CDLL(so_path)
        self.prev = None

    def __enter__(self):
        global _lib
        with _lock:
            self.prev = _lib
            _lib = self.lib
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.prev
        return False


def using(so_path: str) -> _Bound:
    return _Bound(so_path)


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def _dp(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's routines (timing only)."""
    _load().orc_set_threads(ctypes.c_int(int(n)))


def default_angles(n: int) -> np.ndarray:
    """Views evenly spaced over 360 degrees starting at 0."""
    return 2.0 * np.pi * np.arange(n, dtype=np.float64) / n


def matrices(g) -> np.ndarray:
    """[np][3][4] projection matrices acting on (i, j, k, 1) (Section 2.1.1)."""
    lib = _load()
    ang = _f64(g["angles"] if g.get("angles") is not None else default_angles(g["np"]))
    P = np.zeros((g["np"], 3, 4), dtype=np.float64)
    lib.orc_matrices(ctypes.c_double(g["sid"]), ctypes.c_double(g["sdd"]), ctypes.c_int(g["np"]),
                     _dp(ang), ctypes.c_int(g["nu"]), ctypes.c_int(g["nv"]),
                     ctypes.c_double(g["du"]), ctypes.c_double(g["dv"]),
                     ctypes.c_double(g.get("u_off", 0.0)), ctypes.c_double(g.get("v_off", 0.0)),
                     ctypes.c_int(g["nx"]), ctypes.c_int(g["ny"]), ctypes.c_int(g["nz"]),
                     ctypes.c_double(g["sx"]), ctypes.c_double(g["sy"]), ctypes.c_double(g["sz"]),
                     ctypes.c_double(g.get("ox", 0.0)), ctypes.c_double(g.get("oy", 0.0)),
                     ctypes.c_double(g.get("oz", 0.0)), _dp(P))
    return P


def backproject(P, proj, nx, ny, nz, scale=1.0) -> np.ndarray:
    """Listing 1 in double: vol[k][j][i] = scale * sum_s f^2 * bilinear(proj_s, x, y)."""
    lib = _load()
    P = _f64(P)
    q = _f64(proj)
    n_views, nv, nu = q.shape
    vol = np.zeros((nz, ny, nx), dtype=np.float64)
    lib.orc_backproject(_dp(P), ctypes.c_int(n_views), _dp(q), ctypes.c_int(nu), ctypes.c_int(nv),
                        ctypes.c_int(nx), ctypes.c_int(ny), ctypes.c_int(nz),
                        ctypes.c_double(scale), _dp(vol))
    return vol


def backproject_slab(P, proj, nx, ny, k0, nks, scale=1.0) -> np.ndarray:
    """Slices k0..k0+nks-1 of ``backproject`` (same loop and arithmetic)."""
    lib = _load()
    P = _f64(P)
    q = _f64(proj)
    n_views, nv, nu = q.shape
    vol = np.zeros((nks, ny, nx), dtype=np.float64)
    lib.orc_backproject_slab(_dp(P), ctypes.c_int(n_views), _dp(q), ctypes.c_int(nu),
                             ctypes.c_int(nv), ctypes.c_int(nx), ctypes.c_int(ny),
                             ctypes.c_int(k0), ctypes.c_int(nks), ctypes.c_double(scale), _dp(vol))
    return vol


def backproject_points(P, proj, ijk, scale=1.0) -> np.ndarray:
    """``backproject`` evaluated at the voxels listed in ijk ([n][3] of i, j, k)."""
    lib = _load()
    P = _f64(P)
    q = _f64(proj)
    n_views, nv, nu = q.shape
    ijk = np.ascontiguousarray(ijk, dtype=np.int32)
    out = np.zeros(ijk.shape[0], dtype=np.float64)
    lib.orc_backproject_points(_dp(P), ctypes.c_int(n_views), _dp(q), ctypes.c_int(nu),
                               ctypes.c_int(nv), ctypes.c_long(ijk.shape[0]),
                               ijk.ctypes.data_as(_I), ctypes.c_double(scale), _dp(out))
    return out


def forward_project(P, vol, nu, nv, scale=1.0) -> np.ndarray:
    """Exact transpose of ``backproject``: scatter of the same taps and weights."""
    lib = _load()
    P = _f64(P)
    x = _f64(vol)
    nz, ny, nx = x.shape
    n_views = P.shape[0]
    proj = np.zeros((n_views, nv, nu), dtype=np.float64)
    lib.orc_forward_project(_dp(P), ctypes.c_int(n_views), _dp(x), ctypes.c_int(nx), ctypes.c_int(ny),
                            ctypes.c_int(nz), ctypes.c_double(scale), ctypes.c_int(nu),
                            ctypes.c_int(nv), _dp(proj))
    return proj


def mlem(P, proj, nx, ny, nz, iters, subsets=1, x0=None, eps=1e-9) -> np.ndarray:
    """MLEM / ordered-subset EM on the projector pair (scale 1); see orc_mlem."""
    lib = _load()
    P = _f64(P)
    q = _f64(proj)
    n_views, nv, nu = q.shape
    x = np.ones((nz, ny, nx)) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    x = np.ascontiguousarray(x)
    lib.orc_mlem(_dp(P), ctypes.c_int(n_views), _dp(q), ctypes.c_int(nu), ctypes.c_int(nv),
                 ctypes.c_int(nx), ctypes.c_int(ny), ctypes.c_int(nz), ctypes.c_int(subsets),
                 ctypes.c_int(iters), ctypes.c_double(eps), _dp(x))
    return x


def sart(P, proj, nx, ny, nz, iters, subsets=1, lam=1.0, nonneg=False, x0=None, eps=1e-9) -> np.ndarray:
    """Block SART over view subsets (SIRT for one subset); see orc_sart."""
    lib = _load()
    P = _f64(P)
    q = _f64(proj)
    n_views, nv, nu = q.shape
    x = np.zeros((nz, ny, nx)) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    x = np.ascontiguousarray(x)
    lib.orc_sart(_dp(P), ctypes.c_int(n_views), _dp(q), ctypes.c_int(nu), ctypes.c_int(nv),
                 ctypes.c_int(nx), ctypes.c_int(ny), ctypes.c_int(nz), ctypes.c_int(subsets),
                 ctypes.c_int(iters), ctypes.c_double(lam), ctypes.c_int(1 if nonneg else 0),
                 ctypes.c_double(eps), _dp(x))
    return x


def ramp_filter(g, proj) -> np.ndarray:
    """Cosine weight + Ram-Lak, direct linear convolution along u (double)."""
    lib = _load()
    q = _f64(proj)
    n_views, nv, nu = q.shape
    out = np.zeros_like(q)
    lib.orc_filter(ctypes.c_int(n_views), ctypes.c_int(nu), ctypes.c_int(nv),
                   ctypes.c_double(g["du"]), ctypes.c_double(g["dv"]),
                   ctypes.c_double(g.get("u_off", 0.0)), ctypes.c_double(g.get("v_off", 0.0)),
                   ctypes.c_double(g["sid"]), ctypes.c_double(g["sdd"]), _dp(q), _dp(out))
    return out


def ramp_filter_rows(g, proj_rows, r0) -> np.ndarray:
    """``ramp_filter`` for detector rows r0..r0+nr-1 given as [np][nr][nu]."""
    lib = _load()
    q = _f64(proj_rows)
    n_views, nr, nu = q.shape
    out = np.zeros_like(q)
    lib.orc_filter_rows(ctypes.c_int(n_views), ctypes.c_int(nu), ctypes.c_int(g["nv"]),
                        ctypes.c_int(r0), ctypes.c_int(nr),
                        ctypes.c_double(g["du"]), ctypes.c_double(g["dv"]),
                        ctypes.c_double(g.get("u_off", 0.0)), ctypes.c_double(g.get("v_off", 0.0)),
                        ctypes.c_double(g["sid"]), ctypes.c_double(g["sdd"]), _dp(q), _dp(out))
    return out


def phantom_project_rows(g, ellipsoids, r0, nr) -> np.ndarray:
    """``phantom_project`` for detector rows r0..r0+nr-1 ([np][nr][nu])."""
    lib = _load()
    E = _f64(np.asarray(ellipsoids).reshape(-1, 16))
    ang = _f64(g["angles"] if g.get("angles") is not None else default_angles(g["np"]))
    out = np.zeros((g["np"], nr, g["nu"]), dtype=np.float64)
    lib.orc_phantom_project_rows(ctypes.c_double(g["sid"]), ctypes.c_double(g["sdd"]),
                                 ctypes.c_int(g["np"]), _dp(ang), ctypes.c_int(g["nu"]),
                                 ctypes.c_int(g["nv"]), ctypes.c_int(r0), ctypes.c_int(nr),
                                 ctypes.c_double(g["du"]), ctypes.c_double(g["dv"]),
                                 ctypes.c_double(g.get("u_off", 0.0)), ctypes.c_double(g.get("v_off", 0.0)),
                                 ctypes.c_int(E.shape[0]), _dp(E), _dp(out))
    return out


def fdk(g, proj) -> np.ndarray:
    """Feldkamp reconstruction: ramp_filter then backproject with scale pi/np."""
    P = matrices(g)
    Q = ramp_filter(g, proj)
    return backproject(P, Q, g["nx"], g["ny"], g["nz"], scale=np.pi / g["np"])


def phantom_project(g, ellipsoids) -> np.ndarray:
    """Analytic line integrals (density * chord, summed) of an ellipsoid list.

    ellipsoids: [ne][16] rows of cx, cy, cz, ax, ay, az, R (3x3 body->world,
    row-major), rho.
    """
    lib = _load()
    E = _f64(np.asarray(ellipsoids).reshape(-1, 16))
    ang = _f64(g["angles"] if g.get("angles") is not None else default_angles(g["np"]))
    out = np.zeros((g["np"], g["nv"], g["nu"]), dtype=np.float64)
    lib.orc_phantom_project(ctypes.c_double(g["sid"]), ctypes.c_double(g["sdd"]), ctypes.c_int(g["np"]),
                            _dp(ang), ctypes.c_int(g["nu"]), ctypes.c_int(g["nv"]),
                            ctypes.c_double(g["du"]), ctypes.c_double(g["dv"]),
                            ctypes.c_double(g.get("u_off", 0.0)), ctypes.c_double(g.get("v_off", 0.0)),
                            ctypes.c_int(E.shape[0]), _dp(E), _dp(out))
    return out


def siddon(g, vol) -> np.ndarray:
    """Ray-driven line integrals through the piecewise-constant voxel volume."""
    lib = _load()
    x = _f64(vol)
    nz, ny, nx = x.shape
    ang = _f64(g["angles"] if g.get("angles") is not None else default_angles(g["np"]))
    out = np.zeros((g["np"], g["nv"], g["nu"]), dtype=np.float64)
    lib.orc_siddon(ctypes.c_double(g["sid"]), ctypes.c_double(g["sdd"]), ctypes.c_int(g["np"]), _dp(ang),
                   ctypes.c_int(g["nu"]), ctypes.c_int(g["nv"]), ctypes.c_double(g["du"]),
                   ctypes.c_double(g["dv"]), ctypes.c_double(g.get("u_off", 0.0)),
                   ctypes.c_double(g.get("v_off", 0.0)), ctypes.c_int(nx), ctypes.c_int(ny),
                   ctypes.c_int(nz), ctypes.c_double(g["sx"]), ctypes.c_double(g["sy"]),
                   ctypes.c_double(g["sz"]), ctypes.c_double(g.get("ox", 0.0)),
                   ctypes.c_double(g.get("oy", 0.0)), ctypes.c_double(g.get("oz", 0.0)), _dp(x), _dp(out))
    return out


def voxel_centres(g) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """World coordinates (mm) of voxel centres along x, y, z."""
    x = (np.arange(g["nx"]) - 0.5 * (g["nx"] - 1)) * g["sx"] + g.get("ox", 0.0)
    y = (np.arange(g["ny"]) - 0.5 * (g["ny"] - 1)) * g["sy"] + g.get("oy", 0.0)
    z = (np.arange(g["nz"]) - 0.5 * (g["nz"] - 1)) * g["sz"] + g.get("oz", 0.0)
    return x, y, z


# ---------------------------------------------------------------------------
# 3x3x3 convolutions (few-view correction network; no paper counterpart)
# ---------------------------------------------------------------------------

def conv3d(x, w, b=None) -> np.ndarray:
    """Zero-padded 3x3x3 convolution, channels-last: x [N,D,H,W,cin],
    w [cout,27,cin] (tap (dz*3+dy)*3+dx), b [cout] -> y [N,D,H,W,cout]."""
    lib = _load()
    x = _f64(x)
    w = _f64(w)
    N, D, H, W, cin = x.shape
    cout = w.shape[0]
    y = np.zeros((N, D, H, W, cout))
    bp = _dp(_f64(b)) if b is not None else None
    lib.orc_conv3d(_dp(x), N, D, H, W, cin, _dp(w), bp, cout, _dp(y))
    return y


def conv3d_dgrad(dy, w) -> np.ndarray:
    """Input gradient of ``conv3d`` for an output gradient dy [N,D,H,W,cout]."""
    lib = _load()
    dy = _f64(dy)
    w = _f64(w)
    N, D, H, W, cout = dy.shape
    cin = w.shape[2]
    dx = np.zeros((N, D, H, W, cin))
    lib.orc_conv3d_dgrad(_dp(dy), N, D, H, W, cout, _dp(w), cin, _dp(dx))
    return dx


def conv3d_wgrad(x, dy):
    """Weight and bias gradients of ``conv3d``: (dw [cout,27,cin], db [cout])."""
    lib = _load()
    x = _f64(x)
    dy = _f64(dy)
    N, D, H, W, cin = x.shape
    cout = dy.shape[4]
    dw = np.zeros((cout, 27, cin))
    db = np.zeros(cout)
    lib.orc_conv3d_wgrad(_dp(x), _dp(dy), N, D, H, W, cin, cout, _dp(dw), _dp(db))
    return dw, db
