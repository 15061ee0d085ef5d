"""Synthetic antenna arrays (rt_apply_array, Sec. II: plane-wave phases per
element pair after tracing between the array centres) against the FP64
oracle on the same paths, with rotated, dual-polarized devices."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import A_ABS, A_REL, FC, compare_path_sets, gpu_paths, setup

pytestmark = pytest.mark.gpu

LAM = O.C0 / FC


@pytest.fixture(scope="module")
def tracer():
    tr = rt.Tracer(0, FC)
    yield tr
    tr.close()


def _case(tracer, case):
    if case == "tiny_visible":
        sc = S.tiny_scene()
        tx, rx = S.tiny_devices(visible=True)
        N, D = 10000, 2
    else:
        sc = S.city_scene(n_side=6, size=150.0, seed=5)
        tx, rx = S.city_devices(sc, n_rx=24, half=70.0, tx_antenna=S.TR38901_VH)
        rx = S.Devices(rx.pos, rx.ypr + np.float32([0.3, 0.1, -0.2]), S.Antenna(S.ANT_DIPOLE, (np.pi / 4, -np.pi / 4)))
        N, D = 20000, 3
    setup(tracer, sc, tx, rx)
    tracer.compute_paths(D, N)
    gsets, p = gpu_paths(tracer)
    osc = O.make_scene(sc)
    ora_paths, ora_c = O.compute_paths(osc, tx.pos[0], rx.pos, D, N)
    common = compare_path_sets(osc, tx.pos[0], rx.pos, gsets, ora_paths, ora_c)
    sel = [q for q in ora_paths if q.valid]
    return osc, tx, rx, gsets, p["offsets"].cpu().numpy(), sel, common


@pytest.mark.parametrize("case", ["tiny_visible", "small_city"])
def test_array_matches_oracle(tracer, case):
    osc, tx, rx, gsets, off, sel, common = _case(tracer, case)
    tx_el = rt.planar_array(4, 2, 0.7, 0.5, LAM)      # 8 elements, as the paper's example (rows x cols)
    rx_el = rt.planar_array(1, 3, 0.5, 0.5, LAM)
    a, _ = tracer.cir()
    ael = tracer.apply_array(a, tx_el, rx_el).cpu().numpy()
    a = a.cpu().numpy()
    nrp, ntp = a.shape[1], a.shape[2]
    assert ael.shape == (a.shape[0], 3 * nrp, 8 * ntp)
    oa, _ = O.path_field(osc, FC, tx, rx, 0, sel)
    oel = O.array_response(oa, sel, tx.pos[0], tx.ypr[0], rx.pos, rx.ypr, FC, tx_el, rx_el)
    idx = {(q.rx, q.seq): i for i, q in enumerate(sel)}
    n = 0
    for r in range(len(rx.pos)):
        amax = max([np.abs(oa[idx[(r, s)]]).max() for s in common[r]] + [0.0])
        for k, s in enumerate(gsets[r]):
            if s not in common[r]:
                continue
            i, j = off[r] + k, idx[(r, s)]
            err = np.abs(ael[i] - oel[j])
            assert np.all(err <= A_REL * np.abs(oel[j]) + A_ABS * amax), (s, ael[i], oel[j])
            # the array phases alone, on the GPU's own coefficients
            ref = O.array_response(a[i:i + 1].astype(np.complex128), [sel[j]], tx.pos[0], tx.ypr[0], rx.pos,
                                   rx.ypr, FC, tx_el, rx_el)[0]
            assert np.all(np.abs(ael[i] - ref) <= 3e-5 * np.abs(ref) + 1e-7 * amax), (s, ael[i], ref)
            n += 1
    assert n >= 4


def test_array_single_element_and_arguments(tracer):
    _case(tracer, "tiny_visible")
    a, _ = tracer.cir()
    # one element at the centre on both sides: the CIR itself
    assert np.array_equal(tracer.apply_array(a).cpu().numpy(), a.cpu().numpy())
    assert np.array_equal(tracer.apply_array(a, np.zeros((1, 3)), np.zeros((1, 3))).cpu().numpy(), a.cpu().numpy())
    ar = torch.view_as_real(a.contiguous()).contiguous()
    out = torch.empty_like(ar)
    code = rt.lib().rt_apply_array(tracer.ctx, ar.data_ptr(), None, -1, None, 0, out.data_ptr())
    assert code == -1   # RT_ERR_INVALID_ARG
