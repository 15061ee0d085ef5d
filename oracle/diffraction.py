"""FP64 oracle of first-order edge diffraction (Sec. II-B names first-order
diffraction among the features; the paper leaves its equations to the
documentation, so this follows the uniform geometrical theory of
diffraction (UTD) of Kouyoumjian and Pathak for a perfectly conducting
wedge, as stated below).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path. It
shares no code with the CUDA library; occlusion uses the oracle's own
brute-force closest hit.

Wedges: scene edges shared by exactly two triangles whose planes differ.
The solid is taken to be the smaller of the two sectors the faces bound
(convex edges, as the boxes of the synthetic cities have), so the open
exterior angle is n pi with n = 2 - alpha / pi, alpha the angle between the
faces. Face 0 is the triangle with the lower id; angles around the edge are
measured from face 0 through the exterior.

A diffracted path tx -> D -> rx touches the edge at the point D where the
incidence and diffraction angles with the edge agree (Keller's law), which
on the edge line is the point that minimises |tx - D| + |D - rx|. It is
valid when D lies strictly inside the edge, both devices are in the
exterior (0 < phi < n pi), and both segments are free of occluders.

Field of a diffracted path (spherical incidence, ray-fixed coordinates):
  a = lambda/(4 pi) exp(-j k (s' + s)) / sqrt(s s' (s' + s))
      F_rx(-k_d) . [ -D_s b0 b0'^T - D_h p p'^T ] . F_tx(k_i)
with s' = |D - tx|, s = |rx - D|, k_i, k_d the unit incident and diffracted
directions, p' = -(e x k_i)/|.|, b0' = p' x k_i, p = (e x k_d)/|.|,
b0 = p x k_d, and the UTD coefficients
  D_{s,h} = -exp(-j pi/4) / (2 n sqrt(2 pi k) sin b) *
            { cot((pi + (phi - phi'))/(2n)) F(k L a+(phi - phi'))
            + cot((pi - (phi - phi'))/(2n)) F(k L a-(phi - phi'))
            -/+ [ cot((pi + (phi + phi'))/(2n)) F(k L a+(phi + phi'))
                + cot((pi - (phi + phi'))/(2n)) F(k L a-(phi + phi')) ] }
(minus for soft, plus for hard; a term whose cotangent is singular, exactly
on a shadow or reflection boundary, takes the mean of its two one-sided
limits, zero), L = s s' sin^2 b / (s + s'),
a+-(x) = 2 cos^2((2 pi n N+- - x)/2) with N+- the integers nearest to
(x +- pi)/(2 pi n), and the transition function
F(x) = 2 j sqrt(x) exp(j x) int_{sqrt(x)}^inf exp(-j t^2) dt.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.special import fresnel as _fresnel

from . import oracle as O


@dataclass
class Wedge:
    A: np.ndarray       # edge start [3]
    e: np.ndarray       # unit edge direction [3]
    length: float
    f0: int             # face 0 (lower triangle id)
    f1: int
    t0: np.ndarray      # unit vector in face 0, normal to the edge, into the face
    n0: np.ndarray      # unit normal of face 0 on the exterior side
    n: float            # exterior angle / pi


def _inward(A, e, third):
    v = third - A
    v = v - np.dot(v, e) * e
    return v / np.linalg.norm(v)


def wedges(verts: np.ndarray, flat_tol: float = 1e-6) -> list:
    """Wedges of a triangle soup (float32 [T, 9]); edges are matched on the
    exact float32 coordinates of their end points."""
    V = np.asarray(verts, np.float32).reshape(-1, 3, 3)
    table = {}
    for t in range(V.shape[0]):
        for k in range(3):
            p, q = V[t, k], V[t, (k + 1) % 3]
            key = tuple(sorted((tuple(p.tolist()), tuple(q.tolist()))))
            table.setdefault(key, []).append((t, (k + 2) % 3))
    out = []
    for key, faces in table.items():
        if len(faces) != 2:
            continue
        (ta, ka), (tb, kb) = sorted(faces)
        A = np.array(key[0], np.float64)
        B = np.array(key[1], np.float64)
        L = float(np.linalg.norm(B - A))
        if L <= 0.0:
            continue
        e = (B - A) / L
        t0 = _inward(A, e, V[ta, ka].astype(np.float64))
        t1 = _inward(A, e, V[tb, kb].astype(np.float64))
        alpha = float(np.arccos(np.clip(np.dot(t0, t1), -1.0, 1.0)))
        if alpha > np.pi - flat_tol:
            continue   # coplanar faces: no edge
        n0 = np.cross(e, t0)
        if np.dot(n0, t1) > 0.0:
            n0 = -n0
        out.append(Wedge(A, e, L, ta, tb, t0, n0, 2.0 - alpha / np.pi))
    return out


def diffraction_point(w: Wedge, tx, rx):
    """Edge parameter and point of Keller's law on the edge line."""
    tx = np.asarray(tx, np.float64)
    rx = np.asarray(rx, np.float64)
    ts = np.dot(tx - w.A, w.e)
    tr = np.dot(rx - w.A, w.e)
    rs = np.linalg.norm(tx - w.A - ts * w.e)
    rr = np.linalg.norm(rx - w.A - tr * w.e)
    t = ts + (tr - ts) * rs / (rs + rr)
    return t, w.A + t * w.e


def angle(w: Wedge, D, X) -> float:
    """Angle of X around the edge at D, from face 0 through the exterior, in [0, 2 pi)."""
    v = np.asarray(X, np.float64) - D
    return float(np.mod(np.arctan2(np.dot(v, w.n0), np.dot(v, w.t0)), 2.0 * np.pi))


def transition(x: float) -> complex:
    """F(x) = 2 j sqrt(x) exp(j x) int_{sqrt(x)}^inf exp(-j t^2) dt, x >= 0,
    through the normalised Fresnel integrals S, C (scipy)."""
    if x <= 0.0:
        return 0.0 + 0.0j
    u = np.sqrt(x)
    z = u * np.sqrt(2.0 / np.pi)
    S, C = _fresnel(z)
    tail = np.sqrt(np.pi / 2.0) * ((0.5 - C) - 1j * (0.5 - S))
    return 2j * u * np.exp(1j * x) * tail


def _a(x: float, n: float, sign: int) -> float:
    N = np.round((x + sign * np.pi) / (2.0 * np.pi * n))
    return 2.0 * np.cos((2.0 * np.pi * n * N - x) / 2.0) ** 2


def utd_coefficients(n: float, phi: float, phip: float, sin_b: float, s: float, sp: float, k: float):
    """(D_s, D_h) of a perfectly conducting wedge of exterior angle n pi."""
    Lp = s * sp * sin_b ** 2 / (s + sp)
    pre = -np.exp(-1j * np.pi / 4.0) / (2.0 * n * np.sqrt(2.0 * np.pi * k) * sin_b)

    def term(beta, sign):
        arg = (np.pi + sign * beta) / (2.0 * n)
        if abs(np.sin(arg)) < 1e-12:
            # exactly on a shadow or reflection boundary (a set of measure
            # zero): the term's two one-sided limits are +-n sqrt(2 pi k L)
            # exp(j pi/4); their mean, zero, is taken
            return 0.0
        return transition(k * Lp * _a(beta, n, sign)) / np.tan(arg)

    d1 = term(phi - phip, +1) + term(phi - phip, -1)
    d2 = term(phi + phip, +1) + term(phi + phip, -1)
    return pre * (d1 - d2), pre * (d1 + d2)


@dataclass
class DPath:
    rx: int
    wedge: int
    point: np.ndarray
    length: float
    margin: float


def evaluate(osc, w: Wedge, tx, rx):
    """(valid, diffraction point, margin) of the candidate tx -> edge -> rx.
    margin: metres by which a device or the point would have to move to
    change the decision (edge ends, face planes, occluders)."""
    tx = np.asarray(tx, np.float64)
    rx = np.asarray(rx, np.float64)
    t, D = diffraction_point(w, tx, rx)
    m = min(abs(t), abs(w.length - t))
    if not (0.0 < t < w.length):
        return False, D, m
    valid = True
    for X in (tx, rx):
        v = X - D
        r = np.linalg.norm(v - np.dot(v, w.e) * w.e)
        ph = angle(w, D, X)
        m = min(m, r * abs(np.sin(min(ph, abs(w.n * np.pi - ph), np.pi / 2))))
        if not (0.0 < ph < w.n * np.pi):
            valid = False
    if not valid:
        return False, D, m
    for p, q in ((tx, D), (D, rx)):
        clear, mc = O.segment_clear(osc, p, q, w.f0, w.f1)
        m = min(m, mc)
        if not clear:
            valid = False
    # distance from the shadow and reflection boundaries, where one UTD term
    # changes sign (metres at the nearer device)
    pt, pr = angle(w, D, tx), angle(w, D, rx)
    near = min(np.linalg.norm(tx - D), np.linalg.norm(rx - D))
    for beta in (pr - pt, pr + pt):
        for sg in (1.0, -1.0):
            m = min(m, near * 2.0 * w.n * abs(np.sin((np.pi + sg * beta) / (2.0 * w.n))))
    return valid, D, m


def diffracted_paths(osc, scene_verts, tx, rxs, ws=None) -> list:
    """All valid first-order diffracted paths from tx to every receiver."""
    ws = wedges(scene_verts) if ws is None else ws
    tx = np.asarray(tx, np.float64)
    out = []
    for r, rx in enumerate(np.asarray(rxs, np.float64)):
        for wi, w in enumerate(ws):
            ok, D, m = evaluate(osc, w, tx, rx)
            if ok:
                out.append(DPath(r, wi, D, float(np.linalg.norm(D - tx) + np.linalg.norm(rx - D)), m))
    return out


def diffracted_field(ws, paths, fc, txdev, rxdev, tx_index: int = 0):
    """a [P, nrp, ntp] complex128 and tau [P] of diffracted paths."""
    lam = O.C0 / fc
    k = 2.0 * np.pi / lam
    tx = np.asarray(txdev.pos[tx_index], np.float64)
    txa, rxa = txdev.antenna, rxdev.antenna
    a = np.zeros((len(paths), len(rxa.slants), len(txa.slants)), np.complex128)
    tau = np.zeros(len(paths))
    for i, p in enumerate(paths):
        w = ws[p.wedge]
        rx = np.asarray(rxdev.pos[p.rx], np.float64)
        D = p.point
        ki = D - tx
        sp = np.linalg.norm(ki)
        ki /= sp
        kd = rx - D
        s = np.linalg.norm(kd)
        kd /= s
        sin_b = np.linalg.norm(np.cross(w.e, ki))
        pp = -np.cross(w.e, ki)
        pp /= np.linalg.norm(pp)
        bp = np.cross(pp, ki)
        ph = np.cross(w.e, kd)
        ph /= np.linalg.norm(ph)
        bd = np.cross(ph, kd)
        Ds, Dh = utd_coefficients(w.n, angle(w, D, rx), angle(w, D, tx), sin_b, s, sp, k)
        dyad = -Ds * np.outer(bd, bp) - Dh * np.outer(ph, pp)
        amp = lam / (4.0 * np.pi) * np.exp(-1j * k * (s + sp)) / np.sqrt(s * sp * (s + sp))
        for q, zt in enumerate(txa.slants):
            ft = O.antenna(txa.kind, zt, txdev.ypr[tx_index], ki)
            for pr_, zr in enumerate(rxa.slants):
                fr = O.antenna(rxa.kind, zr, rxdev.ypr[p.rx], -kd)
                a[i, pr_, q] = amp * (fr @ dyad @ ft)
        tau[i] = (s + sp) / O.C0
    return a, tau


def diffraction_map(osc, scene_verts, txdev, grid, tx_port: int, rx_antenna, fc: float, ws=None):
    """Diffracted part of a coverage map: per transmitter and cell, the sum of
    |a|^2 (receiver port 0, unrotated, transmit port tx_port) over the
    first-order diffracted paths to the cell centre at grid['h'].
    Returns (gain [n_tx, ny, nx], margin [n_tx, ny, nx]: the smallest decision
    margin of the cell's candidates)."""
    from paper_2303_11103_gb300 import scenes as S   # device records only
    ws = wedges(scene_verts) if ws is None else ws
    nx, ny = int(grid["nx"]), int(grid["ny"])
    gain = np.zeros((len(txdev.pos), ny, nx))
    marg = np.full((len(txdev.pos), ny, nx), np.inf)
    for t in range(len(txdev.pos)):
        tx = S.Devices(txdev.pos[t:t + 1], txdev.ypr[t:t + 1], txdev.antenna)
        for iy in range(ny):
            for ix in range(nx):
                c = np.array([grid["x0"] + (ix + 0.5) * grid["cell"], grid["y0"] + (iy + 0.5) * grid["cell"],
                              grid["h"]], np.float64)
                paths = []
                for wi, w in enumerate(ws):
                    ok, D, m = evaluate(osc, w, tx.pos[0], c)
                    marg[t, iy, ix] = min(marg[t, iy, ix], m)
                    if ok:
                        paths.append(DPath(0, wi, D, 0.0, m))
                if paths:
                    rx = S.Devices(c[None].astype(np.float32), np.zeros((1, 3), np.float32), rx_antenna)
                    a, _ = diffracted_field(ws, paths, fc, tx, rx)
                    gain[t, iy, ix] = float((np.abs(a[:, 0, tx_port]) ** 2).sum())
    return gain, marg
