"""GPU parity of the learned-closure kernels against the FP64 oracle, and the closure's gain.

Inputs and weights are BF16-representable, so the oracle sees exactly the GPU's operands.
Tolerances: FP32-accumulated results 2e-5 relative; BF16-stored outputs within 2^-8 relative
per element (one rounding) plus 1e-6 absolute; AdamW 1e-6 relative.
"""
import numpy as np
import pytest
import torch

from oracle import closure_cnn as ocnn
from oracle import ginzburg_landau as ogl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1708_03188_gb300 import build
    build.build()


def bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


def host(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("cin,cout", [(2, 32), (32, 32), (32, 2)])
def test_conv_layer(cin, cout):
    from paper_1708_03188_gb300 import sgm
    g = np.random.default_rng(cin * 100 + cout)
    B, H, W = 3, 32, 48
    x = bf16(g.standard_normal((B, cin, H, W)))
    w = bf16(g.standard_normal((cout, cin, 3, 3)) * 0.2)
    b = torch.from_numpy(g.standard_normal(cout).astype(np.float32)).cuda()
    xo, wo, bo = host(x), host(w), host(b)
    ref = np.stack([ocnn.conv_forward(xo[i], wo, bo) for i in range(B)])
    y32 = torch.empty((B, cout, H, W), device="cuda")
    sgm.conv3x3_forward(x, w, b, y32, relu=False)
    assert rel(host(y32), ref) < 2e-5
    y16 = torch.empty((B, cout, H, W), dtype=torch.bfloat16, device="cuda")
    sgm.conv3x3_forward(x, w, b, y16, relu=True)
    r = np.maximum(ref, 0)
    assert np.all(np.abs(host(y16) - r) <= 2.0 ** -8 * np.abs(r) + 1e-6)
    # input gradient (with the ReLU mask of a BF16 input) and weight / bias gradients
    gy = torch.from_numpy(g.standard_normal((B, cout, H, W)).astype(np.float32)).cuda()
    gyo = host(gy)
    mask = bf16(np.maximum(g.standard_normal((B, cin, H, W)), 0))
    gx = torch.empty((B, cin, H, W), device="cuda")
    sgm.conv3x3_backward_data(gy, w, mask, gx)
    gx_ref = np.stack([ocnn.conv_backward(xo[i], wo, gyo[i])[0] for i in range(B)]) * (host(mask) > 0)
    assert rel(host(gx), gx_ref) < 2e-5
    gw = torch.zeros((cout, cin, 3, 3), device="cuda")
    gb = torch.zeros(cout, device="cuda")
    sgm.conv3x3_backward_weights(gy, x, gw, gb)
    parts = [ocnn.conv_backward(xo[i], wo, gyo[i]) for i in range(B)]
    assert rel(host(gw), sum(p[1] for p in parts)) < 2e-5
    assert rel(host(gb), sum(p[2] for p in parts)) < 2e-5


def test_network_gradients():
    # the whole network: GPU backward vs the oracle's backward through the same (BF16) activations
    from paper_1708_03188_gb300.closure import ClosureNet
    net = ClosureNet(seed=1)
    g = np.random.default_rng(9)
    B, H, W = 2, 32, 32
    x = bf16(g.standard_normal((B, 2, H, W)))
    out = net.forward(x)
    gout = torch.from_numpy(g.standard_normal(out.shape).astype(np.float32)).cuda()
    net.backward(gout)
    params = [(host(net.Wb[i]), host(net.B[i])) for i in range(4)]
    acts = [host(a) for a in net.acts]
    for i in range(B):
        # oracle forward of the last layer from the GPU's activations
        ref_out = ocnn.conv_forward(acts[3][i], *params[3])
        assert rel(host(out)[i], ref_out) < 2e-5
    grads = [(0.0, 0.0)] * 4
    for i in range(B):
        gi, _ = ocnn.network_backward(params, [a[i] for a in acts] + [host(out)[i]], host(gout)[i])
        grads = [(a + gw, b + gb) for (a, b), (gw, gb) in zip(grads, gi)]
    for li in range(4):
        assert rel(host(net.gW[li]), grads[li][0]) < 1e-4, li
        assert rel(host(net.gB[li]), grads[li][1]) < 1e-4, li


def test_adamw_and_mse():
    from paper_1708_03188_gb300 import sgm
    g = np.random.default_rng(11)
    n = 1000
    w0, gr = g.standard_normal(n), g.standard_normal(n)
    m0, v0 = g.standard_normal(n) * 0.1, np.abs(g.standard_normal(n)) * 0.1
    w = torch.from_numpy(w0.astype(np.float32)).cuda()
    wb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    gt = torch.from_numpy(gr.astype(np.float32)).cuda()
    m = torch.from_numpy(m0.astype(np.float32)).cuda()
    v = torch.from_numpy(v0.astype(np.float32)).cuda()
    sgm.adamw_step(w, wb, gt, m, v, 1e-2, 0.9, 0.999, 1e-8, 1e-4, 7)
    rw, rm, rv = ocnn.adamw_step(host(torch.from_numpy(w0.astype(np.float32))), host(gt), host(torch.from_numpy(
        m0.astype(np.float32))), host(torch.from_numpy(v0.astype(np.float32))), 7, 1e-2, 0.9, 0.999, 1e-8, 1e-4)
    assert rel(host(w), rw) < 1e-6 and rel(host(m), rm) < 1e-6 and rel(host(v), rv) < 1e-6
    assert np.all(host(wb) == host(w.to(torch.bfloat16)))
    out, tgt = torch.randn(777, device="cuda"), torch.randn(777, device="cuda")
    grad, loss = torch.empty_like(out), torch.zeros(1, device="cuda")
    sgm.mse_grad(out, tgt, grad, loss)
    lref, gref = ocnn.mse(host(out), host(tgt))
    assert abs(loss.item() - lref) < 1e-5 * lref and rel(host(grad), gref) < 1e-6


def test_truncate_and_channels():
    from paper_1708_03188_gb300 import sgm
    g = np.random.default_rng(12)
    src = torch.from_numpy((g.standard_normal((2, 48, 48)) + 1j * g.standard_normal((2, 48, 48))).astype(np.complex64)).cuda()
    dst = torch.empty((2, 32, 32), dtype=torch.complex64, device="cuda")
    sgm.spectral_truncate(src, dst)
    for b in range(2):
        assert np.array_equal(dst[b].cpu().numpy(), ogl.truncate(src[b].cpu().numpy(), 32))
    u = src[:, :32, :32].contiguous()
    x = torch.empty((2, 2, 32, 32), dtype=torch.bfloat16, device="cuda")
    sgm.pack_channels(u, x, 2.0)
    assert torch.equal(x[:, 0], (2 * u.real).to(torch.bfloat16)) and torch.equal(x[:, 1], (2 * u.imag).to(torch.bfloat16))
    d = torch.randn((2, 2, 32, 32), device="cuda")
    ref = u + 0.5 * (d[:, 0] + 1j * d[:, 1])
    sgm.unpack_add(d, u, 0.5)
    assert torch.allclose(u, ref, rtol=1e-6, atol=1e-6)


def test_closure_reduces_coarse_error():
    # fine 256^2 truncated to 32^2 (the coarse grid that under-resolves the dynamics at
    # beta = 1.5, gamma = -0.5: plain one-step error ~1e-3), coarse step dt 0.05; trained on 3
    # trajectories, judged on a held-out one: the corrected one-step and 4-step errors must be
    # clearly below the plain ones.
    from paper_1708_03188_gb300 import closure
    coarse = closure.CoarseModel(32, 0.05)
    train_snaps = closure.fine_trajectories(256, 32, 12, 30.0, 30, 0.01, 0.05, first_item=0)
    test_snaps = closure.fine_trajectories(256, 32, 1, 30.0, 20, 0.01, 0.05, first_item=100)
    x, tgt = closure.training_pairs(coarse, train_snaps)
    net = closure.ClosureNet(seed=0)
    hist, scale = closure.train(net, x, tgt, iters=1500, batch=32)
    assert hist[-1] < 0.8 * hist[0], hist
    e_plain, e_learned = closure.relative_errors(coarse, net, test_snaps, scale, horizon=1)
    print("closure one-step errors: plain %.3e learned %.3e; loss %s" % (e_plain, e_learned, hist))
    assert e_learned < 0.8 * e_plain, (e_plain, e_learned)
    e4p, e4l = closure.relative_errors(coarse, net, test_snaps, scale, horizon=4)
    assert e4l < e4p, (e4p, e4l)


def test_fp32_input_layer():
    # the network's first layer reads the FP32 field: forward and weight gradient vs the oracle
    from paper_1708_03188_gb300 import sgm
    g = np.random.default_rng(21)
    B, H, W = 2, 32, 32
    x = torch.from_numpy(g.standard_normal((B, 2, H, W)).astype(np.float32)).cuda()
    w = bf16(g.standard_normal((32, 2, 3, 3)) * 0.3)
    b = torch.zeros(32, device="cuda")
    y = torch.empty((B, 32, H, W), device="cuda")
    sgm.conv3x3_forward(x, w, b, y, relu=False)
    xo, wo = host(x), host(w)
    ref = np.stack([ocnn.conv_forward(xo[i], wo, np.zeros(32)) for i in range(B)])
    assert rel(host(y), ref) < 2e-5
    gy = torch.from_numpy(g.standard_normal((B, 32, H, W)).astype(np.float32)).cuda()
    gw = torch.zeros((32, 2, 3, 3), device="cuda")
    gb = torch.zeros(32, device="cuda")
    sgm.conv3x3_backward_weights(gy, x, gw, gb)
    gref = sum(ocnn.conv_backward(xo[i], wo, host(gy)[i])[1] for i in range(B))
    assert rel(host(gw), gref) < 2e-5


@pytest.mark.parametrize("flags", [0, 1, 2, 4, 7, 6])
def test_augment_pack_matches_the_symmetry_transform(flags):
    """sgm_augment_pack against the same transform in plain torch ops on the gathered pool
    fields: phase, roll by (sx, sy), transposition, reflections (i -> (M - i) mod M), channels."""
    from paper_1708_03188_gb300 import sgm
    g = torch.Generator().manual_seed(7000 + flags)
    n, M, B = 9, 32, 5
    u = torch.complex(torch.randn(n, M, M, generator=g), torch.randn(n, M, M, generator=g)).to(torch.complex64)
    d = torch.complex(torch.randn(n, M, M, generator=g), torch.randn(n, M, M, generator=g)).to(torch.complex64)
    idx = torch.tensor([3, 0, 8, 3, 5], dtype=torch.int32)
    phase = torch.polar(torch.ones(B), torch.rand(B, generator=g) * 6.283185307179586).to(torch.complex64)
    sx, sy, su, sd = 5, 30, 1.0, 2.5
    xu = torch.empty(B, 2, M, M, device="cuda")
    xd = torch.empty_like(xu)
    sgm.augment_pack(u.cuda(), d.cuda(), idx.cuda(), phase.cuda(), sx, sy, flags, su, sd, xu, xd)

    def ref(f, scale):
        v = f[idx.long()].to(torch.complex128) * phase.to(torch.complex128).view(B, 1, 1)
        v = torch.roll(v, (sx, sy), (1, 2))
        if flags & sgm.AUG_TRANSPOSE:
            v = v.transpose(1, 2)
        rev = (-torch.arange(M)) % M
        if flags & sgm.AUG_FLIP0:
            v = v.index_select(1, rev)
        if flags & sgm.AUG_FLIP1:
            v = v.index_select(2, rev)
        return torch.stack([v.real, v.imag], dim=1) * scale

    for got, want in ((xu, ref(u, su)), (xd, ref(d, sd))):
        err = (got.double().cpu() - want).abs().max().item()
        assert err <= 2e-6 * want.abs().max().item()


def test_augment_pack_rejects_bad_arguments():
    from paper_1708_03188_gb300 import sgm
    u = torch.zeros(2, 16, 16, dtype=torch.complex64, device="cuda")
    idx = torch.zeros(3, dtype=torch.int32, device="cuda")
    ph = torch.ones(3, dtype=torch.complex64, device="cuda")
    x = torch.empty(3, 2, 16, 16, device="cuda")
    with pytest.raises(sgm.SgmError):
        sgm.augment_pack(u, u, idx, ph, -1, 0, 0, 1.0, 1.0, x, x.clone())
    with pytest.raises(sgm.SgmError):
        sgm.augment_pack(u, u, idx, ph, 0, 0, 8, 1.0, 1.0, x, x.clone())
