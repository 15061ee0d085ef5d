"""Pins of the CPU surrogate-MLP reference: bfloat16 rounding on known
values, the float64 backward against central finite differences, and the
first Adam step's closed form (lr * g / (|g| + eps))."""
import numpy as np

from oracle import mlp_ref as R


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.0e38, 1e-40], np.float32)
    r = R.to_bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                          # tie -> even mantissa
    assert r[2] == np.float32(1.0 + 2 ** -7)     # above the tie -> up
    assert r[3] == -2.5
    assert np.isfinite(r[4]) or r[4] == np.inf
    assert abs(r[5]) < 1e-39


def _rand_params(F, W, L, rng):
    n = sum((2 * F if l == 0 else W) * (2 if l == L else W) + (2 if l == L else W) for l in range(L + 1))
    p = rng.normal(0, 0.3, n + 6 * F)
    p[n:] = rng.normal(0, 1.0, 6 * F)
    return p


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    F, W, L = 4, 8, 3
    lo, hi = np.full(6, -10.0), np.full(6, 10.0)
    p = _rand_params(F, W, L, rng)
    x = rng.uniform(-10, 10, (16, 6))
    t = np.stack([rng.integers(0, 2, 16), rng.uniform(-140, -60, 16)], 1)
    loss, g = R.loss_and_grads(p, x, t, F, W, L, lo, hi, bf16=False)
    n_train = len(p) - 6 * F
    for k in rng.choice(n_train, 40, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (R.loss_and_grads(pp, x, t, F, W, L, lo, hi, bf16=False)[0] -
              R.loss_and_grads(pm, x, t, F, W, L, lo, hi, bf16=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k]))


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(1)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    new, m, v = R.adam_step(p, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.allclose(p - new, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_friis_baseline_pins():
    """The baseline is the Friis gain: -20 log10(4 pi d / lambda) at 100 m,
    clamped at 1 m, and a loss with the baseline equals the loss on targets
    with the baseline subtracted."""
    lam = 299792458.0 / 3.5e9
    x = np.array([[0, 0, 10, 60, 80, 10], [5, 5, 5, 5, 5, 5.5]], np.float64)
    f = R.friis_db(x, lam)
    assert abs(f[0] - (-20 * np.log10(4 * np.pi * 100.0 / lam))) < 1e-9
    assert abs(f[1] - 20 * np.log10(lam / (4 * np.pi))) < 1e-9
    F, W, L = 4, 64, 2
    lo = np.array([-100, -100, 0, -100, -100, 0.0]); hi = -lo + np.array([0, 0, 20, 0, 0, 20.0])
    rng = np.random.default_rng(3)
    n_p = sum((2 * F if l == 0 else W) * (2 if l == L else W) + (2 if l == L else W) for l in range(L + 1)) + 6 * F
    params = rng.normal(0, 0.1, n_p)
    xs = np.concatenate([rng.uniform(-90, 90, (16, 2)), rng.uniform(5, 15, (16, 1)),
                         rng.uniform(-90, 90, (16, 2)), np.full((16, 1), 1.5)], 1)
    t = np.stack([rng.integers(0, 2, 16).astype(float), rng.uniform(-130, -60, 16)], 1)
    l1, g1 = R.loss_and_grads(params, xs, t, F, W, L, lo, hi, bf16=False, lam=lam)
    t2 = t.copy()
    t2[:, 1] -= R.friis_db(xs, lam)
    l2, g2 = R.loss_and_grads(params, xs, t2, F, W, L, lo, hi, bf16=False, lam=0.0)
    assert abs(l1 - l2) < 1e-12 * max(1.0, abs(l1))
    assert np.allclose(g1, g2, rtol=1e-12, atol=1e-15)
