"""The tcgen05 BF16 GEMM and the warm-start MLP against CPU references: the GEMM against FP64
products of the same BF16 inputs, the MLP's loss and gradients against the FP64 MLP oracle run on
the BF16-rounded weights and inputs."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2203_05027_b300 import build, mfs

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    mfs.load()


def rand_bf16(shape, gen, scale=1.0):
    return (torch.randn(shape, generator=gen) * scale).to(torch.bfloat16)


@pytest.mark.parametrize("M,N,K,splits", [(128, 128, 64, 1), (256, 512, 512, 1), (300, 700, 96, 1),
                                          (64, 200, 32, 1), (256, 512, 4096, 8), (200, 136, 1000, 3)])
def test_gemm_matches_fp64_reference(M, N, K, splits):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A, B = rand_bf16((M, K), g), rand_bf16((N, K), g)
    ref = A.double() @ B.double().T
    Ad, Bd = A.to(dev), B.to(dev)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device=dev)
    mfs.gemm_bf16(M, N, K, Ad.data_ptr(), Bd.data_ptr(), C.data_ptr(), splits=splits,
                  stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    err = (C.cpu().double() - ref).abs().max().item()
    scale = (A.double().abs() @ B.double().abs().T).max().item()
    assert err <= 1e-5 * scale, (err, scale)


def test_gemm_bias_relu_bf16_output():
    M, N, K = 256, 384, 128
    g = torch.Generator().manual_seed(1)
    A, B = rand_bf16((M, K), g), rand_bf16((N, K), g)
    bias = torch.randn(N, generator=g)
    ref = torch.relu(A.double() @ B.double().T + bias.double())
    C = torch.zeros((M, N), dtype=torch.bfloat16, device=dev)
    Ad, Bd, bd = A.to(dev), B.to(dev), bias.to(dev)  # keep the device copies alive during the call
    mfs.gemm_bf16(M, N, K, Ad.data_ptr(), Bd.data_ptr(), C.data_ptr(), bias_ptr=bd.data_ptr(),
                  relu=True, out_fp32=False, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = C.cpu().double()
    assert ((got - ref).abs() <= 1e-2 * ref.abs() + 1e-2).all()
    assert (got[ref == 0] == 0).all()


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("din,width,dout,B", [(32, 64, 200, 16), (32, 512, 700, 64)])
def test_mlp_loss_and_gradients_match_oracle(din, width, dout, B):
    net = mfs.MLP(din, width, dout, max_batch=B, seed=3)
    rng = np.random.default_rng(4)
    mean, std = rng.standard_normal(dout).astype(np.float32), rng.uniform(0.5, 2, dout).astype(np.float32)
    net.set_output_scaling(mean, std)
    X = rng.standard_normal((B, din)).astype(np.float32)
    T = (rng.standard_normal((B, dout)) * 2).astype(np.float32)
    Xd, Td = torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev)
    loss = net.backward(B, Xd.data_ptr(), Td.data_ptr())
    params = [(bf16_round(W), b.astype(np.float64)) for W, b in net.params()]
    grads = net.grads()
    # the oracle keeping the same arrays in BF16 as the device: only accumulation order differs
    oloss, ograds = omlp.loss_and_grads(params, bf16_round(X), T, mean, std, store=bf16_round)
    assert abs(loss - oloss) <= 1e-3 * oloss, (loss, oloss)
    for l, ((gW, gb), (oW, ob)) in enumerate(zip(grads, ograds)):
        assert rel(gW, oW) <= 1e-2, (l, rel(gW, oW))
        assert rel(gb, ob) <= 1e-2, (l, rel(gb, ob))
    # against exact FP64 activations: the effect of BF16 storage stays bounded
    floss, fgrads = omlp.loss_and_grads(params, bf16_round(X), T, mean, std)
    assert abs(loss - floss) <= 1e-2 * floss
    for l, ((gW, gb), (oW, ob)) in enumerate(zip(grads, fgrads)):
        assert rel(gW, oW) <= 1e-1 and rel(gb, ob) <= 1e-1, (l, rel(gW, oW), rel(gb, ob))
    # forward through the same weights
    Y = torch.empty((B, dout), dtype=torch.float32, device=dev)
    net.forward(B, Xd.data_ptr(), Y.data_ptr(), denormalize=True)
    torch.cuda.synchronize()
    oY, _ = omlp.forward(params, bf16_round(X), store=bf16_round)
    assert rel(Y.cpu().numpy(), oY * std + mean) <= 1e-3


def test_mlp_training_reduces_the_loss():
    din, width, dout, B = 32, 128, 300, 64
    net = mfs.MLP(din, width, dout, max_batch=B, seed=5)
    rng = np.random.default_rng(6)
    M = rng.standard_normal((din, dout)) / np.sqrt(din)
    X = rng.standard_normal((B, din)).astype(np.float32)
    T = np.tanh(X @ M).astype(np.float32)
    Xd, Td = torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev)
    first = net.train_step(B, Xd.data_ptr(), Td.data_ptr(), 3e-3)
    for _ in range(200):
        last = net.train_step(B, Xd.data_ptr(), Td.data_ptr(), 3e-3)
    assert last < 0.2 * first, (first, last)


@pytest.mark.parametrize("din,width,dout,B", [(32, 128, 300, 64), (32, 512, 1000, 256), (32, 128, 40, 256)])
def test_fused_train_step_equals_backward_then_adam(din, width, dout, B):
    """train_step computes the output layer inside the GEMM epilogues (loss gradient in the forward
    GEMM, Adam in the weight-gradient GEMM); it must give the same parameters and losses as the
    separate mfs_mlp_backward + mfs_mlp_adam_step path, step after step. In the last case the batch
    has more rows than the output has columns, so the loss GEMM walks its tiles row tile by row
    tile (two row tiles, one column tile)."""
    rng = np.random.default_rng(11)
    X = rng.standard_normal((B, din)).astype(np.float32)
    T = (rng.standard_normal((B, dout)) * 3 + 1).astype(np.float32)
    mean, std = T.mean(0), T.std(0) + 0.1
    Xd, Td = torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev)
    fused, split = mfs.MLP(din, width, dout, B, seed=2), mfs.MLP(din, width, dout, B, seed=2)
    for net in (fused, split):
        net.set_output_scaling(mean, std)
    for step in range(4):
        lf = fused.train_step(B, Xd.data_ptr(), Td.data_ptr(), 1e-3)
        ls = split.backward(B, Xd.data_ptr(), Td.data_ptr())
        split.adam_step(1e-3)
        assert abs(lf - ls) <= 1e-6 * ls, (step, lf, ls)
    for l, ((Wf, bf), (Ws, bs)) in enumerate(zip(fused.params(), split.params())):
        assert rel(Wf, Ws.astype(np.float64)) <= 1e-4, (l, rel(Wf, Ws.astype(np.float64)))
        assert rel(bf, bs.astype(np.float64)) <= 1e-4, l  # rounding differences, amplified by Adam
    # both continue identically from there (the transposed BF16 copy of W3 kept by the fused path)
    Yf = torch.empty((B, dout), device=dev)
    Ys = torch.empty((B, dout), device=dev)
    fused.forward(B, Xd.data_ptr(), Yf.data_ptr())
    split.forward(B, Xd.data_ptr(), Ys.data_ptr())
    torch.cuda.synchronize()
    assert rel(Yf.cpu().numpy(), Ys.cpu().numpy().astype(np.float64)) <= 1e-4


@pytest.mark.parametrize("count,dout", [(1, 9), (700, 133), (20_000, 40)])
def test_fit_output_scaling_matches_fp64_statistics(count, dout):
    g = np.random.default_rng(count + dout)
    # columns with offsets far above their spread (the shifted sums must keep the spread), one
    # constant column (std raised to the floor)
    T = (g.standard_normal((count, dout)) * g.uniform(0.01, 3.0, dout) + g.uniform(-1e3, 1e3, dout)).astype(np.float32)
    T[:, 0] = 5.0
    Td = torch.from_numpy(T).to(dev)
    net = mfs.MLP(8, 32, dout, 16, seed=0)
    net.fit_output_scaling(count, Td.data_ptr(), min_std=1e-3)
    mean, std = net.output_scaling()
    Te = T.astype(np.float64)
    ref_mean, ref_std = Te.mean(0), np.maximum(Te.std(0), 1e-3)
    assert np.allclose(mean, ref_mean, rtol=1e-6, atol=1e-6 * np.abs(ref_mean).max())
    assert np.allclose(std, ref_std, rtol=1e-4, atol=0), np.abs(std / ref_std - 1).max()
    assert std[0] == np.float32(1e-3)
    net.close()


def _f32(x):
    return float(np.float32(x))


def bf16_bits(a):
    """Round-to-nearest-even FP32 -> BF16, as raw 16-bit patterns."""
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16)


@pytest.mark.parametrize("fused", [False, True])
def test_adam_steps_match_oracle(fused):
    """Three optimiser steps against the FP64 Adam oracle (Kingma & Ba), each started from the
    device's own state before the step: FP32 masters, both moments and the BF16 copy, for every
    weight and bias. The hyperparameters are the device's FP32 values promoted to FP64, so only the
    arithmetic differs. fused=True runs mfs_mlp_train_step, where layer 3's update happens in the
    tensor-core GEMM epilogue; its gradient is kept (mfs_mlp_keep_grads) so that the oracle sees the
    same one, and that gradient is itself checked against the FP64 MLP oracle."""
    din, width, dout, B = 32, 128, 200, 64
    net = mfs.MLP(din, width, dout, max_batch=B, seed=7)
    if fused:
        net.keep_grads(True)
    rng = np.random.default_rng(8)
    X = rng.standard_normal((B, din)).astype(np.float32)
    T = (rng.standard_normal((B, dout)) * 2 + 0.5).astype(np.float32)
    mean, std = T.mean(0), T.std(0) + 0.1
    net.set_output_scaling(mean, std)
    Xd, Td = torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev)
    lr = 2e-3
    hp = dict(beta1=_f32(0.9), beta2=_f32(0.999), eps=_f32(1e-8))
    for t in range(1, 4):
        P0 = net.params()
        S0, t0 = net.adam_state()
        assert t0 == t - 1
        if fused:
            net.train_step(B, Xd.data_ptr(), Td.data_ptr(), lr)
        else:
            net.backward(B, Xd.data_ptr(), Td.data_ptr())
            net.adam_step(lr)
        G = net.grads()
        P1 = net.params()
        S1, t1 = net.adam_state()
        assert t1 == t
        if fused and t == 1:
            params = [(bf16_round(W), b.astype(np.float64)) for W, b in P0]
            _, og = omlp.loss_and_grads(params, bf16_round(X), T, mean, std, store=bf16_round)
            assert rel(G[2][0], og[2][0]) <= 1e-2, rel(G[2][0], og[2][0])
        for l in range(3):
            mW0, vW0, mb0, vb0 = S0[l]
            mW1, vW1, mb1, vb1 = S1[l]
            for name, p0, p1, g, m0, m1, v0, v1 in (("W", P0[l][0], P1[l][0], G[l][0], mW0, mW1, vW0, vW1),
                                                     ("b", P0[l][1], P1[l][1], G[l][1], mb0, mb1, vb0, vb1)):
                op, om, ov = omlp.adam_step(p0, g, m0, v0, t, _f32(lr), **hp)
                g64 = np.asarray(g, np.float64)
                mscale = hp["beta1"] * np.abs(m0) + (1 - hp["beta1"]) * np.abs(g64)
                assert (np.abs(m1 - om) <= 1e-6 * mscale + 1e-30).all(), (t, l, name, "m")
                assert (np.abs(v1 - ov) <= 1e-6 * ov + 1e-30).all(), (t, l, name, "v")
                # FP32 rounding of the master weight, plus the FP32 bias corrections 1 - beta^t
                # (cancellation: up to ~3e-5 of the step at t = 2, 3)
                tol = 1e-7 * np.abs(op) + 5e-5 * np.abs(op - p0) + 1e-12
                assert (np.abs(p1 - op) <= tol).all(), (t, l, name, np.abs(p1 - op).max())
                assert np.abs(op - p0).max() > 0.5 * _f32(lr)  # the step moved the parameters
            assert (net.weights_bf16(l) == bf16_bits(P1[l][0])).all(), (t, l)
    net.close()
