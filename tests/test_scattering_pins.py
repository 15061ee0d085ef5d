"""Pins of the first-order diffuse scattering oracle (oracle/scattering.py):
energy balance of the Lambertian pattern over a hemisphere of receivers,
the cos(theta_s) law, and the zero cases (S = 0, receivers behind the
surface or occluded)."""
import numpy as np

from oracle import oracle as O
from oracle import scattering as SC
from paper_2303_11103_gb300 import scenes as S

FC = 3.5e9
LAM = O.C0 / FC


def _patch_scene(extra=None):
    v = np.array([[-1, -1, 0, 1, -1, 0, 1, 1, 0], [-1, -1, 0, 1, 1, 0, -1, 1, 0]], np.float32)
    if extra is not None:
        v = np.concatenate([v, extra.astype(np.float32)])
    return S.Scene(v, np.zeros(len(v), np.int32), np.array([S.CONCRETE], np.float32), "patch")


def _tx():
    return S.Devices(np.array([[0.0, 0.0, 10.0]], np.float32), np.zeros((1, 3), np.float32), S.V_ISO)


def test_isotropic_pattern_has_unit_gain():
    for u in ([1.0, 0.0, 0.0], [0.3, -0.4, 0.866]):
        f = O.antenna(S.ANT_ISO, 0.0, [0.0, 0.0, 0.0], np.array(u) / np.linalg.norm(u))
        assert abs(np.dot(f, f) - 1.0) < 1e-12


def test_lambertian_energy_balance():
    """Receivers on a Fibonacci hemisphere far from a 2 x 2 m patch (S = 1):
    integrating the collected power over the hemisphere returns the scattered
    fraction S^2 (hits / N); the depolarised wave gives a single port half."""
    sc = _patch_scene()
    osc = O.make_scene(sc)
    N = 4000
    hits, _ = O.trace_sbr(osc, _tx().pos[0], N, 1)
    n_hit = int((hits[:, 0] >= 0).sum())
    assert n_hit > 5
    M, Rr = 4000, 3000.0
    d = O.fibonacci(2 * M)
    d = d[d[:, 2] > 0][:M]
    rx = S.Devices((Rr * d).astype(np.float32), np.zeros((len(d), 3), np.float32), S.V_ISO)
    g = SC.scattering_gain(osc, sc.mat_id, np.array([1.0]), FC, _tx(), rx, N)
    power = g[:, 0, 0] * 2.0 * 4 * np.pi * Rr ** 2 / LAM ** 2    # intensity per steradian, both polarisations
    total = power.sum() * (2 * np.pi / len(d))
    assert abs(total - n_hit / N) < 0.01 * n_hit / N


def test_cosine_law_and_zero_cases():
    sc = _patch_scene()
    osc = O.make_scene(sc)
    R = 2000.0
    ang = np.array([0.2, 0.7, 1.2])
    rxp = np.stack([R * np.sin(ang), np.zeros(3), R * np.cos(ang)], 1)
    rxp = np.concatenate([rxp, [[0.0, 0.0, -50.0]]])          # behind the patch
    rx = S.Devices(rxp.astype(np.float32), np.zeros((4, 3), np.float32), S.V_ISO)
    g = SC.scattering_gain(osc, sc.mat_id, np.array([0.6]), FC, _tx(), rx, 3000)[:, 0, 0]
    assert g[0] > 0 and g[3] == 0.0
    for k in (1, 2):
        assert abs(g[k] / g[0] - np.cos(ang[k]) / np.cos(ang[0])) < 2e-3 * np.cos(ang[k]) / np.cos(ang[0])
    # S^2 scaling and S = 0
    g2 = SC.scattering_gain(osc, sc.mat_id, np.array([0.3]), FC, _tx(), rx, 3000)[:, 0, 0]
    assert np.allclose(g2[:3], g[:3] * 0.25, rtol=1e-12)
    assert not SC.scattering_gain(osc, sc.mat_id, np.array([0.0]), FC, _tx(), rx, 3000).any()
    # a wall between the patch and the receiver removes its contribution
    wall = S.box_triangles(30, 31, -20, 20, -5, 40)
    sc2 = _patch_scene(wall)
    osc2 = O.make_scene(sc2)
    rxw = S.Devices(np.array([[100.0, 0.0, 5.0]], np.float32), np.zeros((1, 3), np.float32), S.V_ISO)
    assert SC.scattering_gain(osc2, sc2.mat_id, np.array([1.0]), FC, _tx(), rxw, 3000)[0, 0, 0] == 0.0


def test_vjp_matches_central_differences():
    """The gain is quadratic in every S_m, so central differences of the
    forward oracle are exact up to rounding: they pin the VJP's factor 2 S_m
    and its split over materials (the tiny scene with three materials)."""
    sc = S.tiny_scene_3mat()
    osc = O.make_scene(sc)
    tx = S.Devices(np.array([[-50.0, -50.0, 20.0]], np.float32), np.zeros((1, 3), np.float32), S.TR38901_VH)
    rx = S.Devices(np.array([[-75.0, 0.0, 1.5], [60.0, 10.0, 1.5], [30.0, 25.0, 1.5], [-20.0, -40.0, 6.0]],
                            np.float32), np.zeros((4, 3), np.float32), S.Antenna(S.ANT_DIPOLE, (0.0,)))
    Sm = np.array([0.4, 0.7, 0.25])
    N = 1500
    up = np.random.default_rng(0).normal(size=(4, 1, 2))
    grad = SC.scattering_gain_vjp(osc, sc.mat_id, Sm, FC, tx, rx, N, up)
    h = 1e-3
    fd = np.zeros(3)
    for m in range(3):
        e = np.zeros(3)
        e[m] = h
        gp = SC.scattering_gain(osc, sc.mat_id, Sm + e, FC, tx, rx, N)
        gm = SC.scattering_gain(osc, sc.mat_id, Sm - e, FC, tx, rx, N)
        fd[m] = np.sum(up * (gp - gm)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0 and (np.abs(grad) > 1e-3 * scale).sum() == 3
    assert np.allclose(grad, fd, rtol=1e-8, atol=1e-9 * scale), (grad, fd)


def test_directive_pattern_energy_balance_and_lobe():
    """Directive pattern (alpha_R = 4): over a Fibonacci hemisphere of distant
    receivers the collected power integrates back to S^2 (hits / N), as for
    the Lambertian pattern; the lobe peaks at the specular direction; with
    alpha_R = 0 the intensity is the same in every direction of the
    hemisphere (1 / (2 pi))."""
    sc = _patch_scene()
    osc = O.make_scene(sc)
    tx = S.Devices(np.array([[-6.0, 0.0, 8.0]], np.float32), np.zeros((1, 3), np.float32), S.V_ISO)
    N = 20000
    hits, _ = O.trace_sbr(osc, tx.pos[0], N, 1)
    n_hit = int((hits[:, 0] >= 0).sum())
    assert n_hit > 5
    M, Rr = 4000, 3000.0
    d = O.fibonacci(2 * M)
    d = d[d[:, 2] > 0][:M]
    rx = S.Devices((Rr * d).astype(np.float32), np.zeros((len(d), 3), np.float32), S.V_ISO)
    for a in (0, 4):
        g = SC.scattering_gain(osc, sc.mat_id, np.array([1.0]), FC, tx, rx, N, alpha=[a])
        power = g[:, 0, 0] * 2.0 * 4 * np.pi * Rr ** 2 / LAM ** 2
        total = power.sum() * (2 * np.pi / len(d))
        assert abs(total - n_hit / N) < 0.01 * n_hit / N, (a, total, n_hit / N)
        if a == 0:
            assert np.allclose(power / (n_hit / N), 1.0 / (2 * np.pi), rtol=1e-3)
    # the lobe: receivers on an arc in the plane of incidence; incidence at
    # atan(6/8) from the normal, so the specular direction is 36.87 deg on the +x side
    ang = np.radians(np.arange(-80.0, 81.0, 1.0))
    rxa = S.Devices(np.stack([Rr * np.sin(ang), np.zeros_like(ang), Rr * np.cos(ang)], 1).astype(np.float32),
                    np.zeros((len(ang), 3), np.float32), S.V_ISO)
    g = SC.scattering_gain(osc, sc.mat_id, np.array([1.0]), FC, tx, rxa, 2000, alpha=[6])[:, 0, 0]
    assert abs(np.degrees(ang[np.argmax(g)]) - np.degrees(np.arctan2(6.0, 8.0))) <= 1.0


def test_directive_norm_closed_cases():
    """F_0 is the hemisphere's solid angle 2 pi; F_1 = pi (1 + cos(theta_i) / 2):
    the mean of the integrals of 1 (2 pi) and of k_r . k_s (k_r . pi n)."""
    n = np.array([0.0, 0.0, 1.0])
    for ti in (0.0, 0.4, 1.3):
        kr = np.array([np.sin(ti), 0.0, np.cos(ti)])
        assert abs(SC.directive_norm(0, kr, n) - 2 * np.pi) < 1e-12
        assert abs(SC.directive_norm(1, kr, n) - np.pi * (1 + 0.5 * np.cos(ti))) < 1e-12
