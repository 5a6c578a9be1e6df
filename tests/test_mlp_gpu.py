"""The learned clearance surrogate's tensor-core kernels (tcgen05 BF16 GEMM,
MLP forward / backward / Adam) against numpy and the FP64 oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_10114_gb300 import build, mrs
    build.build()
    mrs.load()


def bf16_bits(x):
    """Round float32 values to bfloat16 (nearest even); bit patterns and values."""
    x = np.ascontiguousarray(x, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    return r, (r.astype(np.uint32) << 16).view(np.float32)


@pytest.mark.parametrize("M,N,K", [(128, 256, 16), (300, 256, 64), (257, 64, 256),
                                   (128, 16, 32), (1000, 256, 4096), (129, 128, 8)])
def test_tcgen05_gemm_matches_numpy(M, N, K):
    from paper_2602_10114_gb300 import mrs
    rng = np.random.default_rng(M + N + K)
    A, Av = bf16_bits(rng.normal(size=(M, K)))
    B, Bv = bf16_bits(rng.normal(size=(N, K)))
    C = mrs.selftest_gemm(A, B)
    ref = Av.astype(np.float64) @ Bv.astype(np.float64).T
    scale = np.abs(Av).astype(np.float64) @ np.abs(Bv).astype(np.float64).T
    assert np.all(np.abs(C - ref) <= 1e-5 * scale + 1e-30)


def _net(in_dim=14, width=256, layers=3, seed=3):
    from paper_2602_10114_gb300 import mrs
    net = mrs.MLP(in_dim, width, layers, seed)
    p = net.get_params()
    # hidden weights exactly representable in BF16, so both sides use the same
    (Ws, (wo, bo)) = net.unpack(p)
    for W, _ in Ws:
        W[:] = bf16_bits(W)[1].reshape(W.shape)
    net.set_params(p)
    return net, p


@pytest.mark.parametrize("over_weight", [1.0, 4.0])
def test_gradients_match_the_fp64_oracle(over_weight):
    """GPU gradients (BF16 GEMMs and activations, FP32 accumulation) against
    the FP64 backward with the same BF16 weights and inputs: 3e-2 relative
    per parameter tensor, cosine > 0.999; plain and asymmetric loss."""
    import torch
    from oracle import oracle as O
    rng = np.random.default_rng(5)
    net, p = _net()
    net.set_loss(over_weight)
    n = 64
    x = bf16_bits(rng.normal(size=(n, 14)))[1]
    t = rng.uniform(-0.15, 0.35, n).astype(np.float32)
    g, loss = net.grads(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    loss_o, g_o, _ = O.mlp_loss_grad(14, 256, 3, p.astype(np.float64), x, t,
                                     over_weight=over_weight)
    assert abs(loss - loss_o) <= 2e-2 * loss_o
    (Ws, (wo, bo)) = net.unpack(g)
    (Wo, (woo, boo)) = net.unpack(g_o)
    pairs = [(a, b) for (Wa, ba), (Wb, bb) in zip(Ws, Wo) for a, b in ((Wa, Wb), (ba, bb))]
    pairs += [(wo, woo), (bo, boo)]
    for a, b in pairs:
        a, b = a.ravel().astype(np.float64), b.ravel().astype(np.float64)
        nb = np.linalg.norm(b)
        if nb == 0:
            assert np.abs(a).max() < 1e-6
            continue
        assert np.linalg.norm(a - b) <= 3e-2 * nb
        assert np.dot(a, b) / (np.linalg.norm(a) * nb) > 0.999


@pytest.mark.parametrize("in_dim,width,layers,rows", [
    (14, 256, 3, 300),      # the self-collision surrogate's shape, a ragged tile
    (14, 256, 3, 5000),     # 40 tiles over the persistent grid
    (20, 48, 2, 257),       # two layer-0 chunks; an odd number of 16-column chunks
    (7, 16, 1, 129),        # one hidden layer of one chunk
    (100, 128, 4, 1000),    # seven layer-0 chunks, four layers
])
def test_forward_matches_the_fp64_oracle(in_dim, width, layers, rows):
    """The fused inference kernel (features, every layer and the output of
    128 rows per CTA) against the FP64 forward with the same BF16 weights and
    inputs; BF16 activations bound the error to about 1e-2 relative."""
    import torch
    from oracle import oracle as O
    rng = np.random.default_rng(6 + rows)
    net, p = _net(in_dim, width, layers)
    x = bf16_bits(rng.normal(size=(rows, in_dim)))[1]
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    _, _, y_o = O.mlp_loss_grad(in_dim, width, layers, p.astype(np.float64), x, np.zeros(rows),
                                False)
    assert np.abs(y - y_o).max() <= 2e-2 * max(1.0, np.abs(y_o).max())


def test_fused_forward_agrees_with_the_training_forward():
    """The training step's layer-by-layer forward and the fused inference
    kernel compute the same network: the loss from the former equals the loss
    of the latter's outputs up to summation order and the fused kernel's
    hardware tanh in SiLU (activation errors of the order of their BF16
    rounding)."""
    import torch
    rng = np.random.default_rng(8)
    net, _ = _net()
    x = rng.uniform(-1, 1, (1000, 14)).astype(np.float32)
    t = rng.uniform(-0.05, 0.25, 1000).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    _, loss = net.grads(xd, td)
    y = net.forward(xd).cpu().numpy().astype(np.float64)
    ref = np.mean((y - np.clip(t, -0.1, 0.3)) ** 2)
    assert abs(loss - ref) <= 1e-2 * ref


def test_adam_training_reduces_the_loss():
    import torch
    rng = np.random.default_rng(7)
    net, _ = _net(seed=11)
    x = rng.uniform(-1, 1, (4096, 14)).astype(np.float32)
    t = (0.1 * np.sin(3 * x[:, 0]) + 0.1 * x[:, 1] * x[:, 2]).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    losses = [net.train_step(xd[i:i + 512], td[i:i + 512], 2e-3)
              for _ in range(40) for i in range(0, 4096, 512)]
    assert np.isfinite(losses).all()
    assert np.mean(losses[-8:]) < 0.6 * np.mean(losses[:8])
