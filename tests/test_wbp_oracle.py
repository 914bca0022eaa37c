"""Pins of the weighted-BP reference (oracle/wbp.py, FP64 autograd):
central finite differences, and equality with the pinned BP oracle when every
weight equals the fixed min-sum scale."""
import numpy as np
import pytest
import torch

from paper_1911_08868_gb300 import inputs


def setup(oracle, N, K, B, seed):
    _, fr = oracle.construct(N, K)
    pay = inputs.payload_numpy(seed, B, K)
    x = oracle.encode_frames(pay, fr, 0, 0)
    llr = inputs.bpsk_awgn_llr(x, inputs.noise_numpy(seed, B, N), inputs.sigma2_of(1.5, K, 0, N))
    return fr, pay, torch.from_numpy(llr.astype(np.float64))


@pytest.mark.parametrize("N,K,T,B", [(16, 8, 3, 3), (64, 32, 2, 2)])
def test_reference_gradient_matches_central_differences(oracle, N, K, T, B):
    from oracle import wbp

    fr, pay, llr = setup(oracle, N, K, B, seed=N)
    n = N.bit_length() - 1
    g = torch.Generator().manual_seed(N)
    w = (0.9375 + 0.05 * torch.randn(T, n, N // 2, 4, generator=g, dtype=torch.float64)).requires_grad_()
    llr = llr.clone().requires_grad_()
    bits = torch.from_numpy(pay)

    def loss(l, ww):
        return wbp.bce_loss(wbp.forward(l, ww, fr, T), bits)

    assert torch.autograd.gradcheck(loss, (llr, w), eps=1e-7, atol=1e-6, rtol=1e-5)


def test_constant_weights_equal_the_bp_oracle(oracle):
    """w = alpha everywhere: the logits are L at level n+1 of the plain
    scaled min-sum decoder (mode 0, no stop) after T iterations."""
    from oracle import wbp

    N, K, T, B = 64, 32, 5, 4
    fr, pay, llr = setup(oracle, N, K, B, seed=3)
    n = N.bit_length() - 1
    w = torch.full((T, n, N // 2, 4), 0.9375, dtype=torch.float64)
    logits = wbp.forward(llr, w, fr, T).numpy()
    s = oracle.Sched(mode=0, stop_kind=0, alpha=0.9375)
    for b in range(B):
        ref = oracle.decode(fr, 0, 0, llr[b].numpy(), s, T, dump=True, dtype=np.float64)
        assert np.array_equal(logits[b], ref.dump[T - 1, 0, n][fr == 0])
