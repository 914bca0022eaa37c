"""Seeded synthetic workloads: random payload bits and a BPSK/AWGN channel.

This module holds no decoder, encoder or code-construction arithmetic; it
only draws the random inputs that both the CUDA path and the CPU oracle
consume, and maps codeword bits to channel LLRs.

Channel (Sec. IV of arXiv 1911.08868): AWGN with QPSK, which with Gray
mapping is two independent BPSK streams at the same per-bit SNR, so BPSK is
simulated.  Energy per bit counts payload bits only (CRC excluded):
sigma^2 = 1 / (2 * R_info * Eb/N0) with R_info = (K - crc_len) / N.  Symbol
s = 1 - 2x, received y = s + sigma * z, LLR = (2 / sigma^2) * y (positive
favours bit 0), all in FP32.
"""
from __future__ import annotations

import numpy as np


def sigma2_of(ebn0_db, K: int, crc_len: int, N: int):
    r_info = (K - crc_len) / N
    return 1.0 / (2.0 * r_info * 10.0 ** (np.asarray(ebn0_db, dtype=np.float64) / 10.0))


def payload_numpy(seed: int, B: int, Kp: int) -> np.ndarray:
    g = np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, 0x5041594C]))
    return g.integers(0, 2, size=(B, Kp), dtype=np.uint8)


def noise_numpy(seed: int, B: int, N: int) -> np.ndarray:
    g = np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, 0x4E4F4953]))
    return g.standard_normal(size=(B, N), dtype=np.float32)


def ebn0_numpy(seed: int, B: int, lo: float, hi: float) -> np.ndarray:
    g = np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, 0x45424E30]))
    return g.uniform(lo, hi, size=B)


def bpsk_awgn_llr(x_bits: np.ndarray, noise: np.ndarray, sigma2) -> np.ndarray:
    """LLRs of codeword bits x (B x N, 0/1) sent as BPSK through AWGN; sigma2 scalar or per row."""
    s2 = np.asarray(sigma2, dtype=np.float64)
    if s2.ndim == 1:
        s2 = s2[:, None]
    sig = np.sqrt(s2).astype(np.float32)
    scale = (2.0 / s2).astype(np.float32)
    s = (1 - 2 * x_bits.astype(np.int8)).astype(np.float32)
    y = s + sig * noise
    return (y * scale).astype(np.float32)


def payload_torch(gen, B: int, Kp: int, device):
    import torch

    return torch.randint(0, 2, (B, Kp), generator=gen, device=device, dtype=torch.uint8)


def bpsk_awgn_llr_torch(x_bits, gen, sigma2):
    """Device twin of bpsk_awgn_llr: noise drawn from the torch generator `gen`."""
    import torch

    B, N = x_bits.shape
    z = torch.randn((B, N), generator=gen, device=x_bits.device, dtype=torch.float32)
    s2 = torch.as_tensor(np.asarray(sigma2, dtype=np.float64), device=x_bits.device)
    if s2.ndim == 1:
        s2 = s2[:, None]
    sig = torch.sqrt(s2).to(torch.float32)
    scale = (2.0 / s2).to(torch.float32)
    s = 1.0 - 2.0 * x_bits.to(torch.float32)
    return (s + sig * z) * scale
