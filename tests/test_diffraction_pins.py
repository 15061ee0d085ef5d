"""Pins of the first-order diffraction oracle (oracle/diffraction.py): wedge
extraction on a box, Keller's law against direct minimisation of the path
length, the transition function against its limits and direct quadrature,
the UTD coefficients against Keller's GTD limit, continuity of the total
field across the incident shadow boundary of a half-plane, and reciprocity."""
import mpmath
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import diffraction as DF
from oracle import oracle as O
from paper_2303_11103_gb300 import scenes as S

FC = 3.5e9
LAM = O.C0 / FC
K0 = 2 * np.pi / LAM


def test_box_wedges():
    """A box has 12 edges, each a 90 degree corner (n = 3/2); the face
    diagonals and a coplanar ground are not edges."""
    v = np.concatenate([S.ground_triangles(100.0), S.box_triangles(-10, 10, -10, 10, 0, 30)]).astype(np.float32)
    ws = DF.wedges(v)
    assert len(ws) == 12
    for w in ws:
        assert abs(w.n - 1.5) < 1e-12
        assert abs(np.dot(w.t0, w.e)) < 1e-12 and abs(np.dot(w.n0, w.e)) < 1e-12
        assert abs(np.dot(w.t0, w.n0)) < 1e-12
    # the exterior normal of face 0 points away from face 1
    for w in ws:
        tri = v[w.f1].reshape(3, 3).astype(np.float64)
        c = tri.mean(0)
        assert np.dot(c - w.A, w.n0) < 0.0


def test_keller_point_minimises_length():
    v = S.box_triangles(-10, 10, -10, 10, 0, 30).astype(np.float32)
    ws = DF.wedges(v)
    rng = np.random.default_rng(3)
    n = 0
    for w in ws:
        for _ in range(5):
            tx = rng.uniform(-40, 40, 3) + np.array([0, 0, 20])
            rx = rng.uniform(-40, 40, 3) + np.array([0, 0, 10])
            t, D = DF.diffraction_point(w, tx, rx)
            f = lambda u: np.linalg.norm(w.A + u * w.e - tx) + np.linalg.norm(rx - w.A - u * w.e)
            best = minimize_scalar(f, bracket=(t - 50, t + 50), tol=1e-12)
            assert abs(best.x - t) < 1e-5
            ki = (D - tx) / np.linalg.norm(D - tx)
            kd = (rx - D) / np.linalg.norm(rx - D)
            assert abs(np.dot(ki, w.e) - np.dot(kd, w.e)) < 1e-12   # equal angles with the edge
            n += 1
    assert n == 60


def test_transition_function():
    # large argument: F -> 1 + j/(2x) - 3/(4x^2)
    for x in (200.0, 1e3, 1e4):
        want = 1 + 0.5j / x - 0.75 / x ** 2
        assert abs(DF.transition(x) - want) < 4.0 / x ** 3
    # small argument: F -> sqrt(pi x) exp(j (pi/4 + x))
    for x in (1e-8, 1e-6):
        want = np.sqrt(np.pi * x) * np.exp(1j * (np.pi / 4 + x))
        assert abs(DF.transition(x) - want) < 3 * x
    # direct quadrature of the definition
    mpmath.mp.dps = 30
    for x in (0.05, 0.7, 3.0, 12.0):
        u = mpmath.sqrt(x)
        tail = mpmath.quadosc(lambda t: mpmath.exp(-1j * t * t), [u, mpmath.inf], zeros=lambda m: mpmath.sqrt(mpmath.pi * m))
        want = complex(2j * u * mpmath.exp(1j * x) * tail)
        assert abs(DF.transition(x) - want) < 1e-9 * max(1.0, abs(want))


def test_utd_reduces_to_gtd():
    """Far from the shadow and reflection boundaries (k L a large) the
    transition functions tend to 1 and the coefficients to Keller's."""
    n, sin_b = 1.5, 0.8
    for phi, phip in [(2.2, 0.6), (3.9, 1.1), (1.3, 0.4)]:
        s = sp = 5e4   # k L ~ 1e6
        Ds, Dh = DF.utd_coefficients(n, phi, phip, sin_b, s, sp, K0)
        # cot((pi+x)/2n) + cot((pi-x)/2n) = 2 sin(pi/n) / (cos(x/n) - cos(pi/n))
        g = np.exp(-1j * np.pi / 4) * np.sin(np.pi / n) / (n * np.sqrt(2 * np.pi * K0) * sin_b)
        c = np.cos(np.pi / n)
        t1 = 1.0 / (c - np.cos((phi - phip) / n))
        t2 = 1.0 / (c - np.cos((phi + phip) / n))
        assert abs(Ds - g * (t1 - t2)) < 1e-4 * abs(g * (t1 - t2))
        assert abs(Dh - g * (t1 + t2)) < 1e-4 * abs(g * (t1 + t2))


@pytest.mark.parametrize("kind", ["soft", "hard"])
def test_half_plane_shadow_boundary_continuity(kind):
    """Half-plane (n = 2), source and observer in a plane normal to the edge:
    the geometrical-optics field switches off at the incident shadow
    boundary phi = pi + phi', and the diffracted field jumps by the same
    amount, so that their sum is continuous. For fields along the
    ray-fixed unit vectors that continue the incident ones (b0 = -b0',
    p = -p' at the boundary) the dyad -D b0 b0' reads u_d = +D u_i A exp(-jks)."""
    n, phip, sp, s = 2.0, 0.7, 40.0, 60.0
    src = sp * np.array([np.cos(phip), np.sin(phip)])
    tot = []
    for dphi in (-2e-4, 2e-4):
        phi = np.pi + phip + dphi
        obs = s * np.array([np.cos(phi), np.sin(phi)])
        Ds, Dh = DF.utd_coefficients(n, phi, phip, 1.0, s, sp, K0)
        D = Ds if kind == "soft" else Dh
        ud = np.exp(-1j * K0 * sp) / sp * D * np.sqrt(sp / (s * (s + sp))) * np.exp(-1j * K0 * s)
        R = np.linalg.norm(obs - src)
        ugo = np.exp(-1j * K0 * R) / R if dphi < 0 else 0.0
        tot.append(ugo + ud)
    assert abs(tot[0] - tot[1]) < 0.02 / (s + sp)


def test_tiny_scene_diffraction_and_reciprocity():
    """Receivers around the tiny scene's box get paths diffracted by its
    vertical edges; with isotropic antennas the coefficients are reciprocal."""
    sc = S.tiny_scene()
    osc = O.make_scene(sc)
    tx, _ = S.tiny_devices(visible=False)
    rx = S.Devices(np.array([[30.0, 25.0, 1.5], [40.0, -30.0, 1.5]], np.float32), np.zeros((2, 3), np.float32), S.V_ISO)
    ws = DF.wedges(sc.verts)
    paths = DF.diffracted_paths(osc, sc.verts, tx.pos[0], rx.pos, ws)
    assert len(paths) >= 2
    a, tau = DF.diffracted_field(ws, paths, FC, tx, rx)
    assert np.all(np.abs(a) > 0)
    for r in range(2):
        mine = [(i, p) for i, p in enumerate(paths) if p.rx == r]
        back = DF.diffracted_paths(osc, sc.verts, rx.pos[r], tx.pos, ws)
        assert sorted(p.wedge for _, p in mine) == sorted(p.wedge for p in back)
        b, taub = DF.diffracted_field(ws, back, FC, S.Devices(rx.pos[r:r + 1], rx.ypr[r:r + 1], rx.antenna), tx)
        for i, p in mine:
            j = [q.wedge for q in back].index(p.wedge)
            assert abs(tau[i] - taub[j]) < 1e-15
            assert abs(a[i, 0, 0] - b[j, 0, 0]) < 1e-9 * abs(a[i, 0, 0])


def test_total_field_continuous_across_shadow_boundary():
    """Full vector pipeline (patterns, ray-fixed bases, dyad): receivers on
    both sides of the shadow boundary of the tiny box's vertical edge at
    (-10, 10). On the lit side the line-of-sight path exists, on the other
    it is blocked; line of sight plus the edge-diffracted path is continuous
    for every port pair."""
    sc = S.tiny_scene()
    osc = O.make_scene(sc)
    ws = DF.wedges(sc.verts)
    wi = [i for i, w in enumerate(ws) if abs(w.e[2]) > 0.99 and np.allclose(w.A[:2], [-10.0, 10.0])]
    assert len(wi) == 1
    tx = S.Devices(np.array([[-60.0, 0.0, 25.0]], np.float32), np.array([[0.2, 0.05, 0.0]], np.float32),
                   S.TR38901_VH)
    y0 = 10.0 * 90.0 / 50.0   # the boundary at x = 30
    tot = []
    for dy in (-2e-5, 2e-5):   # 20 um: the smooth parts barely change across the gap
        rx = S.Devices(np.array([[30.0, y0 + dy, 1.5]], np.float32), np.array([[1.0, 0.0, 0.0]], np.float32),
                       S.Antenna(S.ANT_DIPOLE, (np.pi / 4, -np.pi / 4)))
        dp = [p for p in DF.diffracted_paths(osc, sc.verts, tx.pos[0], rx.pos, ws) if p.wedge == wi[0]]
        assert len(dp) == 1
        ad, _ = DF.diffracted_field(ws, dp, FC, tx, rx)
        los = [p for p in O.compute_paths(osc, tx.pos[0], rx.pos, 0, 0)[0] if p.valid]
        assert len(los) == (1 if dy > 0 else 0)
        al = O.path_field(osc, FC, tx, rx, 0, los)[0].sum(0) if los else 0.0
        tot.append(ad[0] + al)
    scale = LAM / (4 * np.pi * 90.0)
    assert np.all(np.abs(tot[0] - tot[1]) < 0.01 * scale), (tot[0], tot[1])
