"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test ties the oracle to something other than itself: textbook closed
forms (Friis, the two-ray model, Fresnel at normal incidence / Brewster /
grazing, the Snell form of the Fresnel coefficients), Fermat's principle
for image points, reciprocity, exhaustive enumeration on tiny scenes, the
FFT for lattice delays, and central finite differences for the tangents.
"""
import itertools

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import oracle as O
from paper_2303_11103_gb300 import scenes as S

FC = 3.5e9
LAM = O.C0 / FC


def _single_far_triangle_scene():
    """A scene whose only triangle is far away and faces away: free space."""
    v = np.array([[5000, 5000, 5000, 5001, 5000, 5000, 5000, 5001, 5000]], np.float32)
    return S.Scene(v, np.zeros(1, np.int32), np.array([S.CONCRETE], np.float32), "free")


# --------------------------------------------------------------------------- rays
def test_fibonacci_equal_area():
    N = 20000
    d = O.fibonacci(N)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-12)
    # Equal-area: the lattice puts N(1-c)/2 points in every cap {z > c}.
    for c in [-0.9, -0.3, 0.0, 0.45, 0.8]:
        cnt = int((d[:, 2] > c).sum())
        assert abs(cnt - N * (1 - c) / 2) <= 1.0
    # Low discrepancy in azimuth inside a band: each of 8 sectors gets 1/8 of the band.
    band = d[(d[:, 2] > 0.2) & (d[:, 2] < 0.4)]
    phi = np.arctan2(band[:, 1], band[:, 0])
    counts = np.histogram(phi, bins=8, range=(-np.pi, np.pi))[0]
    assert np.all(np.abs(counts - len(band) / 8) < 0.02 * len(band) / 8 + 3)
    # Sub-range queries give the same directions.
    assert np.array_equal(O.fibonacci(N, 1234, 10), d[1234:1244])


def test_closest_hit_ground_and_tie():
    osc = O.make_scene(S.ground_only_scene(100.0))
    i, t, m = O.closest_hit(osc, [3.0, -7.0, 12.5], [0, 0, -1.0])
    assert i in (0, 1) and abs(t - 12.5) < 1e-12 and m > 1.0
    # A ray through the shared diagonal of the ground quad: exact tie -> lowest id, margin 0.
    i, t, m = O.closest_hit(osc, [10.0, 10.0, 5.0], [0, 0, -1.0])
    assert i == 0 and m == 0.0
    # Upward ray misses.
    i, t, m = O.closest_hit(osc, [0, 0, 5.0], [0, 0.6, 0.8])
    assert i == -1 and np.isinf(t)


def test_closest_hit_permutation_invariant():
    rng = np.random.default_rng(7)
    T = 60
    c = rng.uniform(-20, 20, (T, 1, 3))
    V = (c + rng.normal(0, 4, (T, 3, 3))).reshape(T, 9).astype(np.float32)
    sc = S.Scene(V, np.zeros(T, np.int32), np.array([S.CONCRETE], np.float32))
    perm = rng.permutation(T)
    sc2 = S.Scene(V[perm], np.zeros(T, np.int32), sc.materials)
    o1, o2 = O.make_scene(sc), O.make_scene(sc2)
    inv = np.argsort(perm)
    agree = 0
    for _ in range(400):
        o = rng.uniform(-30, 30, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        i1, t1, m1 = O.closest_hit(o1, o, d)
        i2, t2, m2 = O.closest_hit(o2, o, d)
        if m1 < o1.eps:
            continue
        assert (i1 == -1 and i2 == -1) or (i1 == perm[i2] and abs(t1 - t2) < 1e-9)
        agree += i1 >= 0
        # brute-force check of the answer by sampling every triangle
        assert i2 == -1 or inv[i1] == i2
    assert agree > 20


# ------------------------------------------------------------------ image method
def test_image_point_ground_closed_form():
    osc = O.make_scene(S.ground_only_scene(1000.0))
    h1, h2, dist = 25.0, 1.5, 120.0
    tx, rx = [0.0, 0.0, h1], [dist, 0.0, h2]
    ok, pts, length, m = O.image_path(osc, tx, rx, (0,))
    if not ok:
        ok, pts, length, m = O.image_path(osc, tx, rx, (1,))
    assert ok
    assert abs(pts[0, 0] - dist * h1 / (h1 + h2)) < 1e-9 and abs(pts[0, 2]) < 1e-12
    assert abs(length - np.hypot(dist, h1 + h2)) < 1e-9


def test_image_point_fermat_tilted_plane():
    """The reflection point minimises the path length over the plane (Fermat)."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        u = np.cross(n, [0.3, 0.5, 0.8])
        u /= np.linalg.norm(u)
        w = np.cross(n, u)
        c0 = rng.uniform(-5, 5, 3)
        big = 200.0
        quad = [c0 + big * (-u - w), c0 + big * (u - w), c0 + big * (u + w), c0 + big * (-u + w)]
        V = np.array([np.concatenate([quad[0], quad[1], quad[2]]),
                      np.concatenate([quad[0], quad[2], quad[3]])], np.float32)
        osc = O.make_scene(S.Scene(V, np.zeros(2, np.int32), np.array([S.CONCRETE], np.float32)))
        cq = 0.5 * (V[0, :3].astype(np.float64) + V[0, 6:9].astype(np.float64))  # quad centre
        off_t, off_r = rng.uniform(-15, 15, 3), rng.uniform(-15, 15, 3)
        found = False
        for tri in (0, 1):
            Vt = V[tri].astype(np.float64)
            p0 = Vt[:3]
            nn = np.cross(Vt[3:6] - p0, Vt[6:9] - p0)
            nn /= np.linalg.norm(nn)
            tx = cq + off_t
            rx = cq + off_r
            tx = tx + (20 - (tx - p0) @ nn) * nn
            rx = rx + (8 - (rx - p0) @ nn) * nn
            ok, pts, length, m = O.image_path(osc, tx, rx, (tri,))
            if not ok:
                continue
            found = True
            uu = np.cross(nn, [1.0, 0, 0]) if abs(nn[0]) < 0.9 else np.cross(nn, [0, 1.0, 0])
            uu /= np.linalg.norm(uu)
            ww = np.cross(nn, uu)

            def L(q):
                x = p0 + q[0] * uu + q[1] * ww
                return np.linalg.norm(x - tx) + np.linalg.norm(rx - x)

            res = minimize(L, [0.0, 0.0], method="Nelder-Mead",
                           options=dict(xatol=1e-11, fatol=1e-13, maxiter=20000))
            xbest = p0 + res.x[0] * uu + res.x[1] * ww
            assert np.linalg.norm(pts[0] - xbest) < 1e-3
            # a minimum: no point of the plane gives a shorter path
            assert length <= res.fun + 1e-9 and res.fun - length < 1e-5
            # stationarity: equal in-plane components of the two unit directions
            ki = (pts[0] - tx) / np.linalg.norm(pts[0] - tx)
            ko = (rx - pts[0]) / np.linalg.norm(rx - pts[0])
            assert np.linalg.norm((ki - ko) - ((ki - ko) @ nn) * nn) < 1e-9
            assert abs((pts[0] - p0) @ nn) < 1e-9
        assert found


# ------------------------------------------------------------------------ Fresnel
def _snell_fresnel(eps_r, sigma, fc, theta):
    """Textbook Snell form with complex refractive index n2 = sqrt(eta)."""
    eta = eps_r - 1j * sigma / (2 * np.pi * fc * O.EPS0)
    n2 = np.sqrt(eta)
    ci = np.cos(theta)
    ct = np.sqrt(1 - np.sin(theta) ** 2 / eta)
    rs = (ci - n2 * ct) / (ci + n2 * ct)
    rp = (n2 * ci - ct) / (n2 * ci + ct)
    return rs, rp


def test_fresnel_normal_incidence():
    for er, sg in [(5.24, 0.123), (6.31, 0.0036), (2.0, 1.0), (80.0, 4.0)]:
        eta = er - 1j * sg / (2 * np.pi * FC * O.EPS0)
        want = (1 - np.sqrt(eta)) / (1 + np.sqrt(eta))
        rperp, rpar = O.fresnel(er, sg, FC, 1.0)
        assert abs(rperp - want) < 1e-13
        assert abs(rpar + want) < 1e-13   # r_par -> -r_perp: basis flip at normal incidence


def test_fresnel_brewster_and_grazing():
    for er in [2.0, 5.24, 9.0]:
        thb = np.arctan(np.sqrt(er))
        _, rpar = O.fresnel(er, 0.0, FC, np.cos(thb))
        assert abs(rpar) < 1e-12
        rperp, rpar = O.fresnel(er, 0.3, FC, 1e-9)
        assert abs(rperp + 1) < 1e-6 and abs(rpar + 1) < 1e-6


def test_fresnel_matches_snell_form():
    for er, sg in [(5.24, 0.123), (6.31, 0.0036), (3.0, 0.1), (1.5, 0.0)]:
        for th in np.linspace(0.01, 1.55, 17):
            rs, rp = _snell_fresnel(er, sg, FC, th)
            a, b = O.fresnel(er, sg, FC, np.cos(th))
            assert abs(a - rs) < 1e-12 and abs(b - rp) < 1e-12
            if sg == 0.0:
                assert abs(a) <= 1 + 1e-12 and abs(b) <= 1 + 1e-12


# ----------------------------------------------------------------------- antennas
def test_tr38901_pattern_values():
    ypr = [0.0, 0.0, 0.0]
    f = O.antenna(S.ANT_TR38901, 0.0, ypr, [1.0, 0, 0])
    assert abs(10 * np.log10(f @ f) - 8.0) < 1e-12           # boresight: 8 dBi
    assert np.allclose(f / np.linalg.norm(f), [0, 0, -1])    # V-pol = theta_hat
    u = [np.cos(np.radians(65)), np.sin(np.radians(65)), 0]
    f = O.antenna(S.ANT_TR38901, 0.0, ypr, u)
    assert abs(10 * np.log10(f @ f) - (8 - 12)) < 1e-10      # A_H(65 deg) = -12 dB
    f = O.antenna(S.ANT_TR38901, 0.0, ypr, [-1.0, 0, 0])
    assert abs(10 * np.log10(f @ f) - (8 - 30)) < 1e-10      # back lobe floor
    # yaw rotates the boresight, positive pitch tilts it down (TR 38.901 Sec. 7.1)
    f = O.antenna(S.ANT_TR38901, 0.0, [np.pi / 2, 0, 0], [0, 1.0, 0])
    assert abs(10 * np.log10(f @ f) - 8.0) < 1e-10
    p = 0.3
    f = O.antenna(S.ANT_TR38901, np.pi / 2, [0, p, 0], [np.cos(p), 0, -np.sin(p)])
    assert abs(10 * np.log10(f @ f) - 8.0) < 1e-10
    # every pattern vector is transverse to the direction
    rng = np.random.default_rng(0)
    for _ in range(50):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        for kind in (0, 1, 2):
            f = O.antenna(kind, rng.uniform(-1, 1), rng.uniform(-1, 1, 3), u)
            assert abs(f @ u) < 1e-12
    f = O.antenna(S.ANT_DIPOLE, 0.0, ypr, [0, 1.0, 0])
    assert abs(f @ f - 1.5) < 1e-12


# ------------------------------------------------------------- field closed forms
def test_friis_los():
    osc = O.make_scene(_single_far_triangle_scene())
    tx = S.Devices(np.array([[0, 0, 10.0]], np.float32), np.zeros((1, 3), np.float32), S.V_ISO)
    rx = S.Devices(np.array([[173.0, -41.0, 2.0]], np.float32), np.zeros((1, 3), np.float32), S.V_ISO)
    paths, _ = O.compute_paths(osc, tx.pos[0], rx.pos, D=1, N=100)
    assert [p.seq for p in paths] == [()]
    a, tau = O.path_field(osc, FC, tx, rx, 0, paths)
    d = np.linalg.norm(rx.pos[0].astype(np.float64) - tx.pos[0])
    assert abs(abs(a[0, 0, 0]) - LAM / (4 * np.pi * d)) < 1e-12 * LAM / d
    assert abs(tau[0] - d / O.C0) < 1e-18
    # phase = -k0 d modulo 2 pi
    assert abs(np.angle(a[0, 0, 0] * np.exp(2j * np.pi * d / LAM))) < 1e-9
    # TR 38.901 transmitter pointed at the receiver: 8 dBi
    yaw = np.arctan2(-41.0, 173.0)
    pitch = -np.arcsin((2.0 - 10.0) / d)
    txs = S.Devices(tx.pos, np.array([[yaw, pitch, 0]], np.float32), S.TR38901_V)
    a2, _ = O.path_field(osc, FC, txs, rx, 0, paths)
    g = abs(a2[0, 0, 0]) ** 2 / (LAM / (4 * np.pi * d)) ** 2
    assert abs(10 * np.log10(g) - 8.0) < 1e-4


@pytest.mark.parametrize("pol", ["V", "H"])
def test_two_ray_ground(pol):
    eps_r, sigma = S.CONCRETE
    osc = O.make_scene(S.ground_only_scene(2000.0))
    ant = S.Antenna(S.ANT_ISO, (0.0,) if pol == "V" else (np.pi / 2,))
    h1, h2 = 25.0, 1.5
    tx = S.Devices(np.array([[0, 0, h1]], np.float32), np.zeros((1, 3), np.float32), ant)
    dists = np.array([20.0, 75.0, 230.0, 610.0])
    rx = S.Devices(np.stack([dists, np.zeros(4), np.full(4, h2)], 1).astype(np.float32),
                   np.zeros((4, 3), np.float32), ant)
    paths, _ = O.compute_paths(osc, tx.pos[0], rx.pos, D=1, N=20000)
    paths = [p for p in paths if p.valid]
    a, tau = O.path_field(osc, FC, tx, rx, 0, paths)
    k0 = 2 * np.pi / LAM
    for r in range(4):
        idx = [i for i, p in enumerate(paths) if p.rx == r]
        assert len(idx) == 2
        tot = a[idx, 0, 0].sum()
        x = float(rx.pos[r, 0])
        d1 = np.hypot(x, h1 - h2)
        d2 = np.hypot(x, h1 + h2)
        th = np.arctan2(x, h1 + h2)
        rs, rp = _snell_fresnel(eps_r, float(np.float32(sigma)), FC, th)
        if pol == "V":
            want = LAM / (4 * np.pi) * (np.exp(-1j * k0 * d1) / d1 + rp * np.exp(-1j * k0 * d2) / d2)
        else:
            want = -LAM / (4 * np.pi) * (np.exp(-1j * k0 * d1) / d1 + rs * np.exp(-1j * k0 * d2) / d2)
        assert abs(tot - want) < 1e-7 * abs(LAM / (4 * np.pi * d1))


def test_reciprocity_small_city():
    tris = np.concatenate([S.ground_triangles(60.0), S.box_triangles(-5, 5, 8, 20, 0, 12),
                           S.box_triangles(10, 18, -15, -4, 0, 20)])
    sc = S.Scene(tris.astype(np.float32), (np.arange(len(tris)) % 2).astype(np.int32),
                 np.array([S.CONCRETE, S.GLASS], np.float32))
    osc = O.make_scene(sc)
    A = np.array([0.0, 0.0, 9.0])
    B = np.array([8.0, -8.0, 1.5])
    antA = S.Antenna(S.ANT_TR38901, (0.0, np.pi / 2))
    antB = S.Antenna(S.ANT_DIPOLE, (np.pi / 4, -np.pi / 4))
    yA, yB = np.array([[0.4, 0.2, 0.1]]), np.array([[-1.0, 0.05, 0.3]])
    dA = S.Devices(A[None].astype(np.float32), yA.astype(np.float32), antA)
    dB = S.Devices(B[None].astype(np.float32), yB.astype(np.float32), antB)
    pAB = [p for p in O.compute_paths(osc, dA.pos[0], dB.pos, 2, 40000)[0] if p.valid and p.margin > osc.eps]
    pBA = [p for p in O.compute_paths(osc, dB.pos[0], dA.pos, 2, 40000)[0] if p.valid and p.margin > osc.eps]
    sAB = {p.seq for p in pAB}
    sBA = {tuple(reversed(p.seq)) for p in pBA}
    common = sAB & sBA
    assert len(common) >= 5
    aAB, tAB = O.path_field(osc, FC, dA, dB, 0, [p for p in pAB if p.seq in common])
    rev = [p for p in pBA if tuple(reversed(p.seq)) in common]
    rev.sort(key=lambda p: (len(p.seq), tuple(reversed(p.seq))))
    aBA, tBA = O.path_field(osc, FC, dB, dA, 0, rev)
    assert np.allclose(tAB, tBA, rtol=1e-12)
    # swap roles: a_BA[q][p] == a_AB[p][q]
    assert np.allclose(aAB, np.swapaxes(aBA, 1, 2), rtol=1e-9, atol=1e-15)


# ---------------------------------------------------------------- path sets
def test_tiny_scene_is_fully_occluded():
    osc = O.make_scene(S.tiny_scene())
    tx, rx = S.tiny_devices(visible=False)
    paths, _ = O.compute_paths(osc, tx.pos[0], rx.pos, 2, 10000)
    assert [p for p in paths if p.valid] == []
    assert O.brute_force_paths(osc, tx.pos[0], rx.pos[0], 2) == []


def test_tiny_visible_matches_brute_force():
    osc = O.make_scene(S.tiny_scene())
    tx, rx = S.tiny_devices(visible=True)
    paths, _ = O.compute_paths(osc, tx.pos[0], rx.pos, 2, 10000)
    got = sorted(p.seq for p in paths if p.valid)
    bf = sorted(s for s, m in O.brute_force_paths(osc, tx.pos[0], rx.pos[0], 2))
    assert got == bf
    assert len(got) == 4 and () in got
    # closed-form mirror points for the axis-aligned planes
    p = {q.seq: q for q in paths if q.valid}
    wall = [s for s in got if len(s) == 1 and s[0] >= 2][0]
    txp, rxp = np.array([-60.0, 0, 25]), np.array([-75.0, 0, 1.5])
    img = np.array([2 * -10.0 - txp[0], txp[1], txp[2]])          # mirror in x = -10
    s = (-10.0 - rxp[0]) / (img[0] - rxp[0])
    assert np.allclose(p[wall].points[0], rxp + s * (img - rxp), atol=1e-9)
    gnd = [s for s in got if len(s) == 1 and s[0] < 2][0]
    assert abs(p[gnd].points[0, 0] - (-60.0 + (-15.0) * 25.0 / 26.5)) < 1e-9


def test_sbr_subset_of_brute_force_two_boxes():
    tris = np.concatenate([S.ground_triangles(60.0), S.box_triangles(-5, 5, 8, 20, 0, 12),
                           S.box_triangles(10, 18, -15, -4, 0, 20)])
    sc = S.Scene(tris.astype(np.float32), np.zeros(len(tris), np.int32),
                 np.array([S.CONCRETE], np.float32))
    osc = O.make_scene(sc)
    tx = np.array([-20.0, 0.0, 9.0])
    rxs = np.array([[30.0, 2.0, 1.5], [0.0, -25.0, 1.5], [14.0, 10.0, 1.5]])
    paths, _ = O.compute_paths(osc, tx, rxs, 2, 60000)
    for r in range(3):
        got = {p.seq for p in paths if p.valid and p.rx == r}
        bf = {s for s, m in O.brute_force_paths(osc, tx, rxs[r], 2)}
        assert got <= bf
        robust = {s for s, m in O.brute_force_paths(osc, tx, rxs[r], 2) if m > 0.05}
        assert len(robust - got) <= max(1, len(robust) // 10)


# ------------------------------------------------------------------- gradients
def test_dual_tangents_match_central_fd():
    tris = np.concatenate([S.ground_triangles(60.0), S.box_triangles(-5, 5, 8, 20, 0, 12),
                           S.box_triangles(10, 18, -15, -4, 0, 20)])
    mats = np.array([[5.0, 0.01], [3.0, 0.3], [6.5, 0.002], [2.5, 0.8]], np.float32)
    sc = S.Scene(tris.astype(np.float32), (np.arange(len(tris)) % 4).astype(np.int32), mats)
    osc = O.make_scene(sc)
    txd = S.Devices(np.array([[0.0, 0.5, 9.0]], np.float32),
                    np.array([[-0.7, 0.15, 0.05]], np.float32), S.TR38901_VH)
    rxd = S.Devices(np.array([[8.0, -8.0, 1.5], [6.0, 2.0, 1.5]], np.float32),
                    np.array([[0.1, 0, 0], [-0.4, 0.1, 0]], np.float32),
                    S.Antenna(S.ANT_DIPOLE, (0.0, np.pi / 2)))
    paths, _ = O.compute_paths(osc, txd.pos[0], rxd.pos, 2, 20000)
    paths = [p for p in paths if p.valid and p.margin > 0.05]
    assert len(paths) >= 6
    a, tau, da, dtau = O.path_field(osc, FC, txd, rxd, 0, paths, grad=True)
    ng = da.shape[-1]
    assert ng == 6 + 2 * osc.M

    def forward(theta):
        t = np.array(theta, np.float64)
        o2 = O.OScene(osc.V, osc.mat, np.stack([t[6:6 + osc.M], t[6 + osc.M:]], 1), osc.tmin, osc.eps)
        tx2 = S.Devices(t[None, :3], t[None, 3:6], txd.antenna)
        return O.path_field(o2, FC, tx2, rxd, 0, paths)

    theta0 = np.concatenate([txd.pos[0].astype(np.float64), txd.ypr[0].astype(np.float64),
                             osc.mats[:, 0], osc.mats[:, 1]])
    for g in range(ng):
        h = 1e-6 * max(abs(theta0[g]), 1.0)
        tp, tm = theta0.copy(), theta0.copy()
        tp[g] += h
        tm[g] -= h
        ap, taup = forward(tp)
        am, taum = forward(tm)
        fd = (ap - am) / (2 * h)
        fdt = (taup - taum) / (2 * h)
        scale = np.abs(da[..., g]).max() + 1e-30
        assert np.abs(fd - da[..., g]).max() <= 1e-6 * max(scale, np.abs(a).max() * 1e-3)
        assert np.abs(fdt - dtau[:, g]).max() <= 1e-6 * (np.abs(dtau[:, g]).max() + 1e-20)


# ------------------------------------------------------------ frequency response
def test_freq_response_pins():
    f = O.subcarrier_freqs(64, 30e3)
    assert f[0] == -32 * 30e3 and f[32] == 0.0
    a = np.array([0.3 - 0.1j])
    H = O.freq_response(a, np.array([1.234e-6]), f)
    assert np.allclose(np.abs(H), abs(a[0]), rtol=1e-14)
    a2 = np.array([1e-4 + 2e-5j, -3e-5 + 1e-5j])
    t2 = np.array([0.7e-6, 1.9e-6])
    H = O.freq_response(a2, t2, f)
    want = (abs(a2[0]) ** 2 + abs(a2[1]) ** 2 +
            2 * np.real(a2[0] * np.conj(a2[1]) * np.exp(-2j * np.pi * f * (t2[0] - t2[1]))))
    assert np.allclose(np.abs(H) ** 2, want, rtol=1e-12)
    # delays on the lattice n/(K df) reduce to a DFT
    K, df = 128, 30e3
    rng = np.random.default_rng(1)
    n = rng.integers(0, K, 9)
    a3 = rng.normal(size=9) + 1j * rng.normal(size=9)
    H = O.freq_response(a3, n / (K * df), O.subcarrier_freqs(K, df))
    x = np.zeros(K, complex)
    np.add.at(x, n, a3)
    want = np.fft.fft(x) * np.exp(2j * np.pi * (K // 2) * np.arange(K)[None, :] * 0)  # placeholder
    # H[k] = sum_i a_i exp(-j2pi (k-K/2) n_i / K) = X[(k - K/2) mod K]
    X = np.fft.fft(x)
    want = X[(np.arange(K) - K // 2) % K]
    assert np.allclose(H, want, atol=1e-10)


# ------------------------------------------------------------------ coverage map
def _cell_avg_friis(tx, grid, sub=8):
    nx, ny, c = grid["nx"], grid["ny"], grid["cell"]
    xs = grid["x0"] + (np.arange(nx * sub) + 0.5) * c / sub
    ys = grid["y0"] + (np.arange(ny * sub) + 0.5) * c / sub
    X, Y = np.meshgrid(xs, ys)
    r2 = (X - tx[0]) ** 2 + (Y - tx[1]) ** 2 + (grid["h"] - tx[2]) ** 2
    g = (LAM / (4 * np.pi)) ** 2 / r2
    return g.reshape(ny, sub, nx, sub).mean(axis=(1, 3))


def test_coverage_friis_free_space():
    osc = O.make_scene(_single_far_triangle_scene())
    tx = np.array([0.0, 0.0, 10.0])
    grid = dict(x0=-20.0, y0=-20.0, cell=2.0, nx=20, ny=20, h=0.0)
    N = 400000
    g, hits, marg = O.coverage(osc, FC, tx, [0, 0, 0], S.V_ISO, 0, S.V_ISO, N, 0, grid)
    want = _cell_avg_friis(tx, grid)
    # V-pol iso Tx and Rx: polarization match |theta_hat(-d).theta_hat(d)|^2 = 1
    ok = hits >= 16
    assert ok.all()
    rel = np.abs(g - want) / want
    assert np.all(rel < 4.0 / np.sqrt(hits))
    assert np.median(rel) < 0.02


def test_coverage_two_ray_incoherent():
    eps_r, sigma = S.CONCRETE
    osc = O.make_scene(S.ground_only_scene(2000.0))
    tx = np.array([0.0, 0.0, 20.0])
    grid = dict(x0=30.0, y0=-4.0, cell=2.0, nx=10, ny=4, h=1.5)
    N = 2000000
    g, hits, marg = O.coverage(osc, FC, tx, [0, 0, 0], S.V_ISO, 0, S.V_ISO, N, 1, grid)
    xs = grid["x0"] + (np.arange(10) + 0.5) * 2.0
    ys = grid["y0"] + (np.arange(4) + 0.5) * 2.0
    X, Y = np.meshgrid(xs, ys)
    rho = np.hypot(X, Y)
    d1 = np.hypot(rho, 20.0 - 1.5)
    d2 = np.hypot(rho, 20.0 + 1.5)
    th = np.arctan2(rho, 21.5)
    _, rp = _snell_fresnel(eps_r, float(np.float32(sigma)), FC, th)
    want = (LAM / (4 * np.pi)) ** 2 * (1 / d1 ** 2 + np.abs(rp) ** 2 / d2 ** 2)
    rel = np.abs(g - want) / want
    assert np.all(rel < 0.05)
    assert np.median(rel) < 0.02


# ---------------------------------------------------------------- Doppler
def test_doppler_los_closed_forms():
    """LOS: a transmitter closing in on the receiver at v shifts by +v/lambda,
    one moving across the line of sight by 0, a receiver moving away by -v/lambda."""
    osc = O.make_scene(_single_far_triangle_scene())
    tx = np.array([0.0, 0.0, 10.0])
    rx = np.array([[120.0, 0.0, 10.0]])
    paths, _ = O.compute_paths(osc, tx, rx.astype(np.float32), D=1, N=100)
    a = np.array([[[0.3 - 0.4j]]])
    fs, n = 1e6, 14
    t = np.arange(n) / fs
    for vt, vr, fd in [([5.0, 0, 0], None, 5.0 / LAM), ([0, 7.0, 0], None, 0.0),
                       ([0, 0, 0], [[4.0, 0, 0]], -4.0 / LAM), ([3.0, 0, 0], [[3.0, 0, 0]], 0.0)]:
        out = O.doppler(a, paths, tx, rx, FC, fs, n, vt, None if vr is None else np.array(vr))
        assert np.allclose(out[0, 0, 0], a[0, 0, 0] * np.exp(2j * np.pi * fd * t), rtol=1e-12, atol=0)


def test_doppler_ground_reflection_closed_form():
    """Two-ray geometry: the ground path leaves the transmitter at the angle
    theta below the horizon with tan(theta) = (h1 + h2) / d, so a horizontal
    transmitter velocity v towards the receiver shifts it by v cos(theta) / lambda."""
    osc = O.make_scene(S.ground_only_scene(2000.0))
    h1, h2, d = 25.0, 1.5, 230.0
    tx = np.array([0.0, 0.0, h1])
    rx = np.array([[d, 0.0, h2]])
    paths, _ = O.compute_paths(osc, tx, rx.astype(np.float32), D=1, N=20000)
    paths = [p for p in paths if p.valid]
    assert sorted(len(p.seq) for p in paths) == [0, 1]
    a = np.ones((len(paths), 1, 1), complex)
    v = 3.0
    out = O.doppler(a, paths, tx, rx, FC, 1e6, 2, [v, 0.0, 0.0])
    for i, p in enumerate(paths):
        cos_t = d / np.hypot(d, (h1 + h2) if p.seq else (h1 - h2))
        fd = np.angle(out[i, 0, 0, 1]) * 1e6 / (2 * np.pi)
        assert abs(fd - v * cos_t / LAM) < 1e-9 * v / LAM


def test_doppler_is_the_path_length_rate():
    """On a small city the Doppler shift of every valid path equals the rate of
    change of -(path length)/lambda when the devices move (central finite
    difference of the image-method lengths), Fermat's principle for the
    reflection points."""
    tris = np.concatenate([S.ground_triangles(60.0), S.box_triangles(-5, 5, 8, 20, 0, 12),
                           S.box_triangles(10, 18, -15, -4, 0, 20)])
    sc = S.Scene(tris.astype(np.float32), (np.arange(len(tris)) % 2).astype(np.int32),
                 np.array([S.CONCRETE, S.GLASS], np.float32))
    osc = O.make_scene(sc)
    tx = np.array([0.0, 0.0, 9.0])
    rxs = np.array([[8.0, -8.0, 1.5], [-12.0, 3.0, 1.5]])
    paths = [p for p in O.compute_paths(osc, tx, rxs.astype(np.float32), 2, 40000)[0]
             if p.valid and p.margin > osc.eps]
    assert len(paths) >= 5
    vt = np.array([2.0, -1.5, 0.5])
    vr = np.array([[-1.0, 0.7, 0.0], [0.4, 2.0, -0.3]])
    out = O.doppler(np.ones((len(paths), 1, 1), complex), paths, tx, rxs, FC, 1e6, 2, vt, vr)
    h = 1e-3
    for i, p in enumerate(paths):
        ok1, _, l1, _ = O.image_path(osc, tx + h * vt, rxs[p.rx] + h * vr[p.rx], p.seq)
        ok0, _, l0, _ = O.image_path(osc, tx - h * vt, rxs[p.rx] - h * vr[p.rx], p.seq)
        assert ok1 and ok0
        fd_fd = -(l1 - l0) / (2 * h) / LAM
        fd = np.angle(out[i, 0, 0, 1]) * 1e6 / (2 * np.pi)
        assert abs(fd - fd_fd) < 1e-6 * (np.linalg.norm(vt) + 3.0) / LAM, (p.seq, fd, fd_fd)


# ---------------------------------------------------------------- antenna arrays
def _los_paths(tx, rxs):
    osc = O.make_scene(_single_far_triangle_scene())
    paths, _ = O.compute_paths(osc, np.asarray(tx, np.float32), np.asarray(rxs, np.float32), D=1, N=100)
    return paths


def test_array_rotation_is_tr38901():
    """R = Rz(yaw) Ry(pitch) Rx(roll): yaw turns the device x axis towards y,
    positive pitch tilts it downwards (towards -z), and R is orthonormal."""
    R = O.rotation_ypr([np.pi / 2, 0.0, 0.0])
    assert np.allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-15)
    R = O.rotation_ypr([0.0, np.pi / 6, 0.0])
    assert np.allclose(R @ [1, 0, 0], [np.cos(np.pi / 6), 0, -np.sin(np.pi / 6)], atol=1e-15)
    R = O.rotation_ypr([0.3, -0.7, 1.1])
    assert np.allclose(R.T @ R, np.eye(3), atol=1e-14) and abs(np.linalg.det(R) - 1.0) < 1e-14


def test_array_broadside_and_endfire():
    """A linear transmit array along the device y axis: a receiver on the
    boresight (x axis) sees all elements in phase; one along +y sees a phase
    advance of 2 pi d / lambda per element at y = d (that element is closer)."""
    tx = np.array([0.0, 0.0, 10.0])
    rxs = np.array([[300.0, 0.0, 10.0], [0.0, 300.0, 10.0]])
    paths = _los_paths(tx, rxs)
    d = 0.5 * LAM
    tx_el = np.array([[0.0, k * d, 0.0] for k in range(4)])
    a = np.ones((len(paths), 1, 1), complex)
    out = O.array_response(a, paths, tx, [0, 0, 0], rxs, np.zeros((2, 3)), FC, tx_el, np.zeros((1, 3)))
    for i, p in enumerate(paths):
        want = np.ones(4) if p.rx == 0 else np.exp(2j * np.pi * np.arange(4) * d / LAM)
        assert np.allclose(out[i, 0, :], want, atol=1e-12)
    # rotating the device by 90 degrees of yaw swaps the two cases
    out = O.array_response(a, paths, tx, [np.pi / 2, 0, 0], rxs, np.zeros((2, 3)), FC, tx_el, np.zeros((1, 3)))
    for i, p in enumerate(paths):
        want = np.exp(-2j * np.pi * np.arange(4) * d / LAM) if p.rx == 0 else np.ones(4)
        assert np.allclose(out[i, 0, :], want, atol=1e-12)


def test_array_matches_explicit_elements():
    """Against explicit modelling on a small city (Sec. II: paths traced for
    every element): the exact image-method length from each displaced element
    pair gives exp(-j 2 pi (L_mn - L_00) / lambda), which the plane-wave phase
    matches to within the curvature error pi (|r| + |s|)^2 / (lambda L)."""
    tris = np.concatenate([S.ground_triangles(60.0), S.box_triangles(-5, 5, 8, 20, 0, 12),
                           S.box_triangles(10, 18, -15, -4, 0, 20)])
    sc = S.Scene(tris.astype(np.float32), (np.arange(len(tris)) % 2).astype(np.int32),
                 np.array([S.CONCRETE, S.GLASS], np.float32))
    osc = O.make_scene(sc)
    tx = np.array([0.0, 0.0, 9.0])
    rxs = np.array([[8.0, -8.0, 1.5], [-12.0, 3.0, 1.5]])
    txy, rxy = np.array([0.4, 0.1, 0.2]), np.array([[-1.0, 0.0, 0.3], [2.0, 0.05, -0.1]])
    paths = [p for p in O.compute_paths(osc, tx, rxs.astype(np.float32), 2, 40000)[0]
             if p.valid and p.margin > osc.eps]
    assert len(paths) >= 5
    d = 0.5 * LAM
    tx_el = np.array([[0.0, c * d, r * 0.7 * LAM] for r in (-0.5, 0.5) for c in (-0.5, 0.5)])
    rx_el = np.array([[0.0, c * d, 0.0] for c in (-0.5, 0.5)])
    a = np.ones((len(paths), 1, 1), complex)
    out = O.array_response(a, paths, tx, txy, rxs, rxy, FC, tx_el, rx_el)
    Rt = O.rotation_ypr(txy)
    for i, p in enumerate(paths):
        Rr = O.rotation_ypr(rxy[p.rx])
        ok, _, L0, _ = O.image_path(osc, tx, rxs[p.rx], p.seq)
        assert ok
        bound = 2 * np.pi * (np.linalg.norm(tx_el, axis=1).max() + np.linalg.norm(rx_el, axis=1).max()) ** 2 / (LAM * L0)
        for n in range(len(rx_el)):
            for m in range(len(tx_el)):
                ok, _, L, _ = O.image_path(osc, tx + Rt @ tx_el[m], rxs[p.rx] + Rr @ rx_el[n], p.seq)
                assert ok
                exact = np.exp(-2j * np.pi * (L - L0) / LAM)
                assert abs(np.angle(out[i, n, m] / exact)) < bound, (p.seq, n, m)
