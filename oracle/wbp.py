"""Weighted BP reference (TEST INFRASTRUCTURE ONLY): plain PyTorch CPU ops in FP64.

Unrolled round-trip BP on the original (unpermuted) polar factor graph of
Sec. II-B with the scaled min-sum f of the paper, except that every f
evaluation has its own learnable scale: w[t, s, q, k] for iteration t,
stage s (0-based, counted from the channel), processing element q of that
stage (pairing t = q with a zero inserted at bit n-1-s, and b = t + 2^(n-1-s)),
and k indexing the PE's four f evaluations:
    k = 0: L_out1 = f(L_in1, L_in2 + R_in2)
    k = 1: L_out2 = f(R_in1, L_in1) + L_in2
    k = 2: R_out1 = f(R_in1, L_in2 + R_in2)
    k = 3: R_out2 = f(R_in1, L_in1) + R_in2
f_w(a, b) = w * sign(a) sign(b) * min(|a|, |b|); when |a| == |b| the first
operand is taken as the minimum (the gradient goes to a); near a = 0 with a
the minimum, f_w = w a sign(b), whose derivative w sign(b) is used at 0 too.  The logits are
L at level n+1 on the information positions after T iterations (the last R
sweep does not reach them and is not run).  Frozen priors are a large
finite number (1e200) instead of +inf, so that autograd never forms
0 * inf; no message ever reaches that magnitude otherwise, and +inf and
1e200 select the same minimum everywhere.

Autograd of this function is the gradient reference; it is pinned by
central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np
import torch

BIG = 1e200      # frozen prior in FP64
BIG32 = 1e30     # frozen prior in FP32 (products with weights and sums stay finite)


def pe_pairs(n: int, s: int):
    """(t, b) index tensors of the N/2 processing elements of stage s."""
    N = 1 << n
    p = n - 1 - s
    q = torch.arange(N // 2)
    t = ((q >> p) << (p + 1)) | (q & ((1 << p) - 1))
    return t, t | (1 << p)


def f_w(a, b, w):
    # w * sign(a) sign(b) min(|a|, |b|), written as w * a sign(b) when a is
    # the minimum (else w * b sign(a)) so that autograd has the true
    # derivative w sign(b) at a = 0 (R messages fed by information priors are
    # exactly 0); the sign factors carry no gradient.
    return w * torch.where(a.abs() <= b.abs(), a * torch.sign(b), b * torch.sign(a))


def forward(llr: torch.Tensor, w: torch.Tensor, frozen: np.ndarray, T: int) -> torch.Tensor:
    """llr [B, N], w [T, n, N/2, 4] (float64, or float32 for FP32 comparisons) -> logits [B, K]."""
    B, N = llr.shape
    n = N.bit_length() - 1
    fr = torch.as_tensor(np.asarray(frozen, dtype=bool))
    big = BIG if llr.dtype == torch.float64 else BIG32
    prior = torch.where(fr, torch.tensor(big, dtype=llr.dtype), torch.tensor(0.0, dtype=llr.dtype))
    prior = prior.expand(B, N)
    zeros = torch.zeros(B, N, dtype=llr.dtype)
    R = [zeros] * (n + 1)                      # R[l-1] = R at level l
    R[n] = prior
    for it in range(T):
        L = [llr] + [None] * n
        for s in range(n):
            t, b = pe_pairs(n, s)
            Lin, Rin = L[s], R[s + 1]
            out = torch.zeros(B, N, dtype=llr.dtype)
            out = out.index_put((torch.arange(B)[:, None], t[None, :]),
                                f_w(Lin[:, t], Lin[:, b] + Rin[:, b], w[it, s, :, 0]))
            out = out.index_put((torch.arange(B)[:, None], b[None, :]),
                                f_w(Rin[:, t], Lin[:, t], w[it, s, :, 1]) + Lin[:, b])
            L[s + 1] = out
        if it == T - 1:
            break
        Rn = list(R)
        for s in range(n - 1, 0, -1):           # stage 0 only produces R at level 1 (unused)
            t, b = pe_pairs(n, s)
            Lin, Rin = L[s], Rn[s + 1]
            out = torch.zeros(B, N, dtype=llr.dtype)
            out = out.index_put((torch.arange(B)[:, None], t[None, :]),
                                f_w(Rin[:, t], Lin[:, b] + Rin[:, b], w[it, s, :, 2]))
            out = out.index_put((torch.arange(B)[:, None], b[None, :]),
                                f_w(Rin[:, t], Lin[:, t], w[it, s, :, 3]) + Rin[:, b])
            Rn[s] = out
        R = Rn
    info = torch.as_tensor(np.nonzero(~np.asarray(frozen, dtype=bool))[0])
    return L[n][:, info]


def bce_loss(logits: torch.Tensor, bits: torch.Tensor) -> torch.Tensor:
    """Mean binary cross-entropy of the information bits; a positive logit favours bit 0."""
    return torch.nn.functional.binary_cross_entropy_with_logits(-logits, bits.to(logits.dtype))
