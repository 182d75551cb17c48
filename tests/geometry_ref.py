"""Independent vector-geometry restatement of the circular cone-beam setup.

Used by the oracle's pins: it projects points by intersecting the ray from
the source with the detector plane, instead of applying a 3x4 matrix, so a
mistake in the matrix construction (a sign, a transposed term, a missing
offset) shows up as a disagreement. Conventions (our reading of Section
2.1.1, which skips the derivation): source at sid*e_r, detector plane normal
to e_r at distance sdd from the source, e_u = (-sin t, cos t, 0),
e_v = (0, 0, 1), pixel centres at integer indices.
"""
import numpy as np


def frame(theta):
    er = np.array([np.cos(theta), np.sin(theta), 0.0])
    eu = np.array([-np.sin(theta), np.cos(theta), 0.0])
    ev = np.array([0.0, 0.0, 1.0])
    return er, eu, ev


def voxel_world(g, i, j, k):
    return np.array([(i - 0.5 * (g["nx"] - 1)) * g["sx"] + g.get("ox", 0.0),
                     (j - 0.5 * (g["ny"] - 1)) * g["sy"] + g.get("oy", 0.0),
                     (k - 0.5 * (g["nz"] - 1)) * g["sz"] + g.get("oz", 0.0)])


def project_point(g, theta, X):
    """(u, v, w): detector pixel coordinates hit by the ray source->X, and the
    ratio of X's depth along the central ray to sid."""
    er, eu, ev = frame(theta)
    S = g["sid"] * er
    O = S - g["sdd"] * er          # detector centre point (foot of the central ray)
    d = X - S
    t = np.dot(O - S, er) / np.dot(d, er)
    H = S + t * d
    U = np.dot(H - O, eu)
    V = np.dot(H - O, ev)
    cu = 0.5 * (g["nu"] - 1) + g.get("u_off", 0.0)
    cv = 0.5 * (g["nv"] - 1) + g.get("v_off", 0.0)
    w = np.dot(S - X, er) / g["sid"]
    return U / g["du"] + cu, V / g["dv"] + cv, w


def pixel_ray(g, theta, r, c):
    """Source position and unit direction of the ray through pixel (r, c)."""
    er, eu, ev = frame(theta)
    S = g["sid"] * er
    O = S - g["sdd"] * er
    cu = 0.5 * (g["nu"] - 1) + g.get("u_off", 0.0)
    cv = 0.5 * (g["nv"] - 1) + g.get("v_off", 0.0)
    Pix = O + (c - cu) * g["du"] * eu + (r - cv) * g["dv"] * ev
    d = Pix - S
    return S, d / np.linalg.norm(d)
