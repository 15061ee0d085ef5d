"""compute_paths sizes its candidate hash table from the previous call's key
count and reads the count only after the hash pass. A table that turns out
too small (the device counts more keys than it holds) is detected on the
device and the pass is repeated with the count read back. Either way the
candidates and paths must be those of a fresh context."""
import numpy as np
import pytest
import torch

from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _run(tr, rays):
    P = tr.compute_paths(3, rays)
    p = tr.paths()
    tx, dep, seq, wit = tr.candidates()
    return P, {k: v.cpu().numpy() for k, v in p.items()}, (tx.cpu().numpy(), dep.cpu().numpy(), seq.cpu().numpy(),
                                                            wit.cpu().numpy())


def _same(a, b):
    Pa, pa, ca = a
    Pb, pb, cb = b
    assert Pa == Pb
    for k in ("offsets", "seq", "depth"):
        assert np.array_equal(pa[k], pb[k]), k
    assert np.array_equal(pa["length"], pb["length"])
    for x, y in zip(ca, cb):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("order", [(4_000, 200_000), (200_000, 4_000)])
def test_hash_table_sized_by_an_earlier_call(order):
    sc = S.city_scene(n_side=6, size=150.0, seed=5)
    tx, rx = S.city_devices(sc, n_rx=64, seed=3, half=70.0)
    small, large = order
    tr = rt.Tracer(0, 3.5e9)
    tr.load_scene(sc)
    tr.set_devices(tx, rx)
    _run(tr, small)                 # sizes the table for the next call
    got = _run(tr, large)           # larger key count: overflow and repeat; smaller: fits
    again = _run(tr, large)         # sized by the call before: fits
    fresh = rt.Tracer(0, 3.5e9)
    fresh.load_scene(sc)
    fresh.set_devices(tx, rx)
    want = _run(fresh, large)
    _same(got, want)
    _same(again, want)
    torch.cuda.synchronize()
    tr.close()
    fresh.close()
