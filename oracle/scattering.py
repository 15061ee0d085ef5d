"""FP64 oracle of first-order diffuse scattering (Sec. II-B lists diffuse
reflections, i.e. scattering, among the features and leaves the model to
the documentation; the reading here is the effective-roughness model with a
Lambertian pattern).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path. It
shares no code with the CUDA library; hits and occlusion use the oracle's
brute-force closest hit and segment test.

Each of the N Fibonacci-lattice rays of a transmitter carries the fraction
|F_tx,q(d)|^2 / N of the transmitted power (its solid angle 4 pi / N). Where
it first hits a surface of scattering coefficient S, the fraction S^2 of
that power is re-radiated with the Lambertian intensity pattern
cos(theta_s) / pi on the side the ray came from. A receiver at distance r
from the hit point in that half-space, with the segment to it unoccluded,
collects with the effective aperture lambda^2 / (4 pi) |F_rx,p|^2, and the
scattered wave is taken as depolarised, so a single-polarised port
receives half of it:
  g[p][q] += S^2 (|F_tx,q(d)|^2 / N) (cos theta_s / pi)
             (lambda^2 / (4 pi r^2)) |F_rx,p(-k_s)|^2 / 2.
The result is the incoherent scattered path gain of every (tx, rx) pair and
port pair. The specular coefficients are left as they are.

Scattering pattern per material: alpha < 0 takes the Lambertian pattern
above; alpha >= 0 the directive pattern of the effective-roughness model, a
lobe around the specular direction k_r:
  intensity(k_s) = ((1 + k_r . k_s) / 2)^alpha / F_alpha,
with F_alpha the integral of the lobe over the hemisphere on the incident
side (here by Gauss-Legendre quadrature in cos(theta_s) and the trapezoidal
rule in azimuth, both exact for this polynomial integrand), so that the
pattern re-radiates exactly the fraction S^2 like the Lambertian one.

Gradients with respect to the scattering coefficients (Sec. II names the
parameters of the scattering functions among the differentiable inputs):
the gain is S_m^2 times the gain the rays hitting material m would carry at
S_m = 1, so dL/dS_m = 2 S_m sum(dL/dg * g_m(S_m = 1)).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def directive_norm(alpha: int, kr, n, n_mu: int = 40) -> float:
    """F_alpha: integral of ((1 + kr . k_s)/2)^alpha over the unit vectors k_s
    with k_s . n > 0 (cos(theta_s) by Gauss-Legendre, azimuth by the
    trapezoidal rule; the integrand is a polynomial of degree alpha)."""
    n = np.asarray(n, np.float64)
    e1 = np.cross(n, [1.0, 0.0, 0.0] if abs(n[0]) < 0.9 else [0.0, 1.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    x, wx = np.polynomial.legendre.leggauss(n_mu)
    mu, wmu = 0.5 * (x + 1.0), 0.5 * wx
    n_phi = 2 * n_mu
    phi = 2.0 * np.pi * np.arange(n_phi) / n_phi
    st = np.sqrt(1.0 - mu ** 2)
    ks = (st[:, None, None] * (np.cos(phi)[None, :, None] * e1 + np.sin(phi)[None, :, None] * e2)
          + mu[:, None, None] * n)
    f = ((1.0 + ks @ np.asarray(kr, np.float64)) / 2.0) ** alpha
    return float((f * wmu[:, None]).sum() * (2.0 * np.pi / n_phi))


def scattering_gain(osc, scene_mat, S, fc: float, txdev, rxdev, N: int, ray_ids=None, tx_index: int = 0,
                    alpha=None):
    """g [R, nrp, ntp]: incoherent first-order scattered gain from transmitter
    tx_index to every receiver, over the lattice rays ray_ids (all N when None;
    each ray keeps the weight 1/N). scene_mat: int [T] material ids; S [M];
    alpha [M] pattern per material (None: all Lambertian)."""
    lam = O.C0 / fc
    tx = np.asarray(txdev.pos[tx_index], np.float64)
    txa, rxa = txdev.antenna, rxdev.antenna
    R = len(rxdev.pos)
    g = np.zeros((R, len(rxa.slants), len(txa.slants)))
    ids = np.arange(N) if ray_ids is None else np.asarray(ray_ids)
    dirs = O.fibonacci(N)
    for i in ids:
        d = dirs[i]
        j, t, _ = O.closest_hit(osc, tx, d, -1)
        if j < 0:
            continue
        s = float(S[int(scene_mat[j])])
        if s <= 0.0:
            continue
        V = osc.V[j].reshape(3, 3)
        n = np.cross(V[1] - V[0], V[2] - V[0])
        n /= np.linalg.norm(n)
        if np.dot(d, n) > 0.0:
            n = -n          # the side the ray came from
        P = tx + t * d
        a_m = -1 if alpha is None else int(alpha[int(scene_mat[j])])
        if a_m >= 0:
            kr = d - 2.0 * np.dot(d, n) * n          # specular direction
            F = directive_norm(a_m, kr, n)
        ptx = np.array([np.dot(O.antenna(txa.kind, z, txdev.ypr[tx_index], d),
                               O.antenna(txa.kind, z, txdev.ypr[tx_index], d)) for z in txa.slants])
        for r in range(R):
            rx = np.asarray(rxdev.pos[r], np.float64)
            v = rx - P
            dist = np.linalg.norm(v)
            cs = np.dot(v, n) / dist
            if cs <= 0.0:
                continue
            clear, _ = O.segment_clear(osc, P, rx, j, -1)
            if not clear:
                continue
            ks = v / dist
            prx = np.array([np.dot(O.antenna(rxa.kind, z, rxdev.ypr[r], -ks),
                                   O.antenna(rxa.kind, z, rxdev.ypr[r], -ks)) for z in rxa.slants])
            pattern = cs / np.pi if a_m < 0 else ((1.0 + np.dot(kr, ks)) / 2.0) ** a_m / F
            w = s * s / N * pattern * lam ** 2 / (4.0 * np.pi * dist ** 2) * 0.5
            g[r] += w * np.outer(prx, ptx)
    return g


def scattering_gain_vjp(osc, scene_mat, S, fc: float, txdev, rxdev, N: int, up, tx_index: int = 0, alpha=None):
    """dL/dS [M] from the upstream gradient up [R, nrp, ntp] of scattering_gain,
    by the derivative of the definition: one unit-coefficient run per material."""
    S = np.asarray(S, np.float64)
    grad = np.zeros(len(S))
    for m in range(len(S)):
        if S[m] <= 0.0:     # S <= 0 scatters nothing (as in scattering_gain)
            continue
        one = np.zeros(len(S))
        one[m] = 1.0
        gm = scattering_gain(osc, scene_mat, one, fc, txdev, rxdev, N, tx_index=tx_index, alpha=alpha)
        grad[m] = 2.0 * S[m] * float(np.sum(np.asarray(up) * gm))
    return grad
