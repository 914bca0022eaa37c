"""Weighted BP kernels through the C ABI against the FP64 autograd reference
(oracle/wbp.py): FP64 kernels match it (values exactly, gradients to
rounding), torch.autograd.gradcheck passes on the FP64 kernels, FP32 kernels
agree within FP32 tolerance, and a short training run lowers the loss."""
import numpy as np
import pytest
import torch

from paper_1911_08868_gb300 import inputs

from conftest import gpu_device

pytestmark = pytest.mark.gpu


def setup(oracle, N, K, B, T, seed, ebn0=1.5):
    _, fr = oracle.construct(N, K)
    pay = inputs.payload_numpy(seed, B, K)
    x = oracle.encode_frames(pay, fr, 0, 0)
    llr = inputs.bpsk_awgn_llr(x, inputs.noise_numpy(seed, B, N), inputs.sigma2_of(ebn0, K, 0, N))
    n = N.bit_length() - 1
    g = torch.Generator().manual_seed(seed)
    w = 0.9375 + 0.05 * torch.randn(T, n, N // 2, 4, generator=g, dtype=torch.float64)
    return fr, torch.from_numpy(pay), torch.from_numpy(llr.astype(np.float64)), w


def reference(fr, pay, llr, w, T):
    from oracle import wbp

    l = llr.clone().requires_grad_()
    ww = w.clone().requires_grad_()
    logits = wbp.forward(l, ww, fr, T)
    loss = wbp.bce_loss(logits, pay)
    loss.backward()
    return logits.detach(), ww.grad, l.grad


def gpu_run(pcbp, code, llr, w, pay, T, dtype):
    from oracle import wbp

    dev = gpu_device()
    l = llr.to(dev, dtype).requires_grad_()
    ww = w.to(dev, dtype).requires_grad_()
    logits = pcbp.wbp(l, ww, code, T)
    loss = wbp.bce_loss(logits, pay.to(dev))
    loss.backward()
    torch.cuda.synchronize()
    return logits.detach().cpu().double(), ww.grad.cpu().double(), l.grad.cpu().double()


@pytest.mark.parametrize("N,K,T,B", [(16, 8, 4, 5), (64, 32, 5, 7), (256, 128, 3, 9)])
def test_fp64_kernels_match_reference(pcbp, oracle, N, K, T, B):
    fr, pay, llr, w = setup(oracle, N, K, B, T, seed=N + T)
    code = pcbp.pc_construct(N, K)
    rl, rw, rg = reference(fr, pay, llr, w, T)
    gl, gw, gg = gpu_run(pcbp, code, llr, w, pay, T, torch.float64)
    assert torch.equal(gl, rl)
    assert torch.allclose(gw, rw, rtol=1e-10, atol=1e-14)
    assert torch.allclose(gg, rg, rtol=1e-10, atol=1e-14)
    assert rw.abs().sum() > 0


@pytest.mark.parametrize("N,K,T,B", [(16, 8, 3, 2), (64, 32, 2, 2)])
def test_gradcheck_fp64_kernels(pcbp, oracle, N, K, T, B):
    fr, pay, llr, w = setup(oracle, N, K, B, T, seed=7 * N)
    code = pcbp.pc_construct(N, K)
    dev = gpu_device()
    l = llr.to(dev).requires_grad_()
    ww = w.to(dev).requires_grad_()
    bits = pay.to(dev)
    from oracle import wbp

    def loss(a, b):
        return wbp.bce_loss(pcbp.wbp(a, b, code, T), bits)

    assert torch.autograd.gradcheck(loss, (l, ww), eps=1e-7, atol=1e-6, rtol=1e-5)


@pytest.mark.parametrize("case", [(32, 16, 6, 40), (256, 128, 10, 64), (1024, 512, 6, 24),
                                  (256, 128, 4, 1000), (1024, 512, 3, 400), (128, 64, 5, 300),
                                  (512, 256, 4, 160)],
                         ids=lambda c: f"N{c[0]}-B{c[3]}")
def test_fp32_kernels_match_fp32_reference(pcbp, oracle, case):
    """FP32 kernels against the same reference evaluated in FP32: identical
    operation order, so the logits match exactly and the gradients differ
    only in summation order.  Against FP64, min-sum near-ties resolve
    differently in a few processing elements (the gradient is rerouted), so
    that comparison is loose.  The larger batches give every frame slot several
    frames in turn."""
    N, K, T, B = case
    fr, pay, llr, w = setup(oracle, N, K, B, T, seed=99)
    code = pcbp.pc_construct(N, K)
    r32l, r32w, r32g = reference(fr, pay, llr.float(), w.float(), T)
    gl, gw, gg = gpu_run(pcbp, code, llr.float(), w.float(), pay, T, torch.float32)
    assert torch.equal(gl, r32l.double())
    assert (gw - r32w.double()).norm() / r32w.double().norm() < 1e-4
    assert (gg - r32g.double()).norm() / r32g.double().norm() < 1e-4
    if N == 256:
        r64l, r64w, _ = reference(fr, pay, llr, w, T)
        assert (gl - r64l).abs().max() / r64l.abs().max() < 1e-3
        assert (gw - r64w).norm() / r64w.norm() < 2e-2


def test_training_lowers_the_loss(pcbp, oracle):
    """A few Adam steps on frames made by pc_encode and the AWGN channel."""
    from oracle import wbp

    dev = gpu_device()
    N, K, T, B = 64, 32, 5, 512
    code = pcbp.pc_construct(N, K)
    n = N.bit_length() - 1
    w = torch.full((T, n, N // 2, 4), 0.9375, device=dev, requires_grad=True)
    opt = torch.optim.Adam([w], lr=0.02)
    gen = torch.Generator(device=dev).manual_seed(5)
    losses = []
    for step in range(25):
        pay = inputs.payload_torch(gen, B, K, dev)
        x = torch.empty((B, N), dtype=torch.uint8, device=dev)
        pcbp.pc_encode(code, pay, x)
        llr = inputs.bpsk_awgn_llr_torch(x, gen, inputs.sigma2_of(2.0, K, 0, N)).contiguous()
        loss = wbp.bce_loss(pcbp.wbp(llr, w, code, T), pay)
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert np.mean(losses[-5:]) < np.mean(losses[:5])


@pytest.mark.parametrize("N,K", [(64, 32), (1024, 512)])
def test_fp32_unaligned_checkpoint_buffer(pcbp, oracle, N, K):
    """The unrolled FP32 forward writes its checkpoint rows as float4 into a 16-byte aligned buffer
    and one float at a time otherwise; both give the backward the same checkpoints: identical
    logits and LLR gradients, the weight gradient equal up to the order of its atomic sums."""
    T, B = 4, 48
    fr, pay, llr, w = setup(oracle, N, K, B, T, seed=5 * N)
    code = pcbp.pc_construct(N, K)
    dev = gpu_device()
    l = llr.to(dev, torch.float32).contiguous()
    ww = w.to(dev, torch.float32).contiguous()
    cnt = pcbp.wbp_ckpt_count(code, T, B)
    ws = torch.empty(pcbp.wbp_workspace_size(code, T, B, 4), dtype=torch.uint8, device=dev)
    gl = (torch.randn((B, K), generator=torch.Generator().manual_seed(3)) * 1e-2).to(dev)
    out = []
    for off in (0, 1):                         # off = 1: the buffer starts 4 bytes past a 16-byte boundary
        store = torch.zeros(cnt + 4, dtype=torch.float32, device=dev)
        ckpt = store[off:off + cnt]
        logits = torch.empty((B, K), dtype=torch.float32, device=dev)
        pcbp.wbp_forward(code, l, ww, T, logits, ckpt, ws)
        gw = torch.zeros_like(ww)
        gllr = torch.empty_like(l)
        pcbp.wbp_backward(code, l, ww, T, ckpt, gl, gw, gllr, ws)
        torch.cuda.synchronize()
        out.append((logits.cpu(), gllr.cpu(), gw.cpu().double()))
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
    assert (out[0][2] - out[1][2]).norm() <= 1e-5 * out[0][2].norm()
    assert out[0][2].abs().sum() > 0
