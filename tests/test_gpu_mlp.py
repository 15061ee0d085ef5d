"""tcgen05 BF16 GEMM and the surrogate MLP's training / inference kernels.

The GEMM is compared with a plain PyTorch FP32 matmul of the same BF16
inputs; the MLP's loss, gradients and Adam update with the CPU reference
(oracle/mlp_ref.py) that rounds to BF16 at the same points."""
import numpy as np
import pytest
import torch

from oracle import mlp_ref as R
from paper_2303_11103_gb300 import rt

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (200, 256, 256), (256, 64, 1000), (384, 128, 512),
                                   (1, 8, 8), (1000, 192, 256)])
def test_gemm_matches_fp32_reference(M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ref = A.float() @ B.float().T
    C = rt.rt_gemm_bf16(A, B, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    err = (C - ref).abs().max().item()
    assert err <= 1e-4 * ref.abs().max().item() + 1e-4
    C2 = rt.rt_gemm_bf16(A, B, bias=bias, relu=True, out_bf16=True, status=status)
    ref2 = torch.relu(ref + bias)
    assert torch.allclose(C2.float(), ref2, rtol=1e-2, atol=1e-2 * ref2.abs().max().item())


def _surrogate(seed=3):
    lo = np.array([-250, -250, 0, -250, -250, 0], np.float32)
    hi = np.array([250, 250, 100, 250, 250, 10], np.float32)
    return rt.Surrogate(lo, hi, n_freq=32, width=256, n_hidden=8, sigma=2.0, seed=seed), lo, hi


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    x = np.concatenate([rng.uniform(-250, 250, (n, 2)), rng.uniform(20, 80, (n, 1)),
                        rng.uniform(-250, 250, (n, 2)), np.full((n, 1), 1.5)], 1).astype(np.float32)
    d = np.linalg.norm(x[:, :3] - x[:, 3:], axis=1)
    gain = -20 * np.log10(4 * np.pi * d / 0.0857) + 3 * np.sin(x[:, 3] / 30)
    has = (np.sin(x[:, 0] / 40) + np.cos(x[:, 4] / 25) > -0.5).astype(np.float32)
    return x, np.stack([has, gain], 1).astype(np.float32)


@pytest.mark.parametrize("lam", [0.0, 299792458.0 / 3.5e9])
def test_mlp_gradients_match_reference(lam):
    S, lo, hi = _surrogate()
    S.set_baseline(lam)
    x, t = _batch(256, 0)
    p0 = S.params().cpu().numpy().astype(np.float64)
    loss = torch.zeros(1, device="cuda")
    S.train_step(torch.as_tensor(x).cuda(), torch.as_tensor(t).cuda(), 1e-3, loss)
    g_gpu = S.grads().cpu().numpy()
    p1 = S.params().cpu().numpy()
    torch.cuda.synchronize()
    assert S.status() == 0
    ref_loss, g_ref = R.loss_and_grads(p0.astype(np.float32), x, t, S.F, S.W, S.L, lo, hi, bf16=True, lam=lam)
    assert abs(loss.item() - ref_loss) <= 2e-3 * abs(ref_loss)
    # per layer: relative L2 error of the gradient at BF16 tolerance
    o = 0
    for l in range(S.L + 1):
        fi = 2 * S.F if l == 0 else S.W
        fo = 2 if l == S.L else S.W
        for n in (fi * fo, fo):
            a, b = g_gpu[o:o + n], g_ref[o:o + n]
            assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-12, (l, n)
            o += n
    # the Adam update applied to the reference gradient reproduces the new parameters
    p_ref, _, _ = R.adam_step(p0, g_gpu.astype(np.float64), np.zeros_like(p0), np.zeros_like(p0), 1, 1e-3)
    assert np.allclose(p1, p_ref, rtol=1e-5, atol=1e-7)
    S.close()


def test_mlp_inference_matches_reference_and_learns():
    S, lo, hi = _surrogate(seed=5)
    x, t = _batch(4096, 1)
    xt, tt = torch.as_tensor(x).cuda(), torch.as_tensor(t).cuda()
    losses = []
    for it in range(300):
        loss = torch.zeros(1, device="cuda")
        S.train_step(xt[(it % 8) * 512:(it % 8 + 1) * 512], tt[(it % 8) * 512:(it % 8 + 1) * 512], 1e-3, loss)
        losses.append(loss.item())
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:5])
    # fused all-layer kernel == layer-by-layer GEMMs (same BF16 rounding points)
    big = torch.cat([xt] * 3)[:10007]                    # several tiles per CTA, ragged tail
    fused = S.infer(big)
    layered = S.infer_layers(big)
    torch.cuda.synchronize()
    assert S.status() == 0
    assert torch.allclose(fused, layered, rtol=1e-4, atol=1e-3)
    out = S.infer(xt[:777]).cpu().numpy()             # ragged count
    p = S.params().cpu().numpy()
    y, _, _, _ = R.forward(p, x[:777], S.F, S.W, S.L, lo, hi, bf16=True)
    assert np.allclose(out[:, 0], y[:, 0], rtol=2e-2, atol=2e-2)
    assert np.allclose(out[:, 1], y[:, 1] * R.DB_SCALE + R.DB_OFFSET, rtol=2e-3, atol=0.2)
    S.close()


def test_baseline_outputs_match_reference():
    """With the free-space baseline the fused kernel, the layer-by-layer path
    and the CPU reference give the same gain output (residual + Friis)."""
    S, lo, hi = _surrogate(seed=9)
    lam = 299792458.0 / 3.5e9
    S.set_baseline(lam)
    x, _ = _batch(1000, 4)
    xt = torch.as_tensor(x).cuda()
    fused = S.infer(xt)
    layered = S.infer_layers(xt)
    torch.cuda.synchronize()
    assert torch.allclose(fused, layered, rtol=1e-4, atol=1e-3)
    p = S.params().cpu().numpy()
    y, _, _, _ = R.forward(p, x, S.F, S.W, S.L, lo, hi, bf16=True)
    assert np.allclose(fused.cpu().numpy()[:, 1], R.gain_db(y, x, lam), rtol=2e-3, atol=0.2)
    with pytest.raises(rt.RtError):
        S.set_baseline(-1.0)
    S.close()


def test_surrogate_save_load_roundtrip():
    """rt_mlp_save / rt_mlp_load: a trained model, saved and loaded into a
    new model, answers bit for bit as the original; a corrupted buffer is
    rejected."""
    S, lo, hi = _surrogate(seed=5)
    S.set_baseline(299792458.0 / 3.5e9)
    x, t = _batch(512, 3)
    xd, td = torch.as_tensor(x).cuda(), torch.as_tensor(t).cuda()
    for _ in range(3):
        S.train_step(xd, td, 1e-3)
    q, _ = _batch(1000, 4)
    qd = torch.as_tensor(q).cuda()
    y0 = S.infer(qd)
    data = S.save()
    S2 = rt.Surrogate.load(data)
    assert (S2.F, S2.W, S2.L, S2.n_params) == (S.F, S.W, S.L, S.n_params)
    assert torch.equal(S2.params(), S.params())
    assert torch.equal(S2.infer(qd), y0)
    assert torch.equal(S2.infer_layers(qd), S.infer_layers(qd))
    assert S2.save() == data
    bad = bytearray(data)
    bad[200] ^= 1
    with pytest.raises(rt.RtError):
        rt.Surrogate.load(bytes(bad))
    S.close()
    S2.close()
