"""A library built with PCBP_CHECKED=1 range-checks every shared-memory plane
access, TMEM column, channel-LLR index and decision-word index of the
tensor-memory decoder kernel and records any access out of range in a status
word of the workspace (redirecting the access, so nothing faults).  On such a
build these tests decode a spread of lengths, schedules and event shapes and
require that no access was out of range; on a normal build they are skipped."""
import numpy as np
import pytest

from conftest import gpu_device
from test_gpu_parity import DECODE_CASES, KERNEL_CASES, POLY8, POLY24, frames

pytestmark = pytest.mark.gpu

EXTRA = [
    # permuted stages narrower than a group (single-stage path), every N of the kernel
    (128, 64, 8, POLY8, 1.5, dict(mode=1, P_range=2, P_level=6, N_min=1, T0=1), 40, 300),
    (256, 128, 8, POLY8, 1.5, dict(mode=1, P_range=2, P_level=7, N_min=1, T0=1, stop_kind=3), 40, 300),
    (512, 256, 24, POLY24, 1.5, dict(mode=1, P_range=2, P_level=8, N_min=1, T0=1), 40, 300),
    (2048, 1024, 24, POLY24, 1.5, dict(mode=1, P_range=2, P_level=10, N_min=1, T0=1, stop_kind=2), 30, 200),
    # full-order events (FP-BP) and every event shape drawn at random
    (2048, 1024, 24, POLY24, 2.0, dict(mode=2, it_reset_full=2, q_max=0), 30, 200),
    (1024, 512, 24, POLY24, 2.0, dict(mode=1, P_range=10, P_level=9, N_min=1, T0=1, fkind=1, alpha=1.0), 30, 200),
]


def status_of(dec) -> int:
    return int.from_bytes(bytes(dec.workspace[16:20].cpu().tolist()), "little")


@pytest.mark.parametrize("case", DECODE_CASES + KERNEL_CASES + EXTRA,
                         ids=lambda c: f"N{c[0]}-mode{c[5]['mode']}-f{c[5].get('fkind', 0)}-s{c[5].get('stop_kind', 1)}")
def test_no_access_out_of_range(pcbp, oracle, case):
    import torch

    if not pcbp.build_checked():
        pytest.skip("not a bounds-checked build (PCBP_CHECKED=1)")
    dev = gpu_device()
    N, K, r, poly, ebn0, kw, max_iters, B = case
    _, _, _, llr = frames(oracle, N, K, r, poly, B, ebn0, seed=N * 5 + kw["mode"])
    s = pcbp.sched(**{"seed": 31, "stop_kind": 1, **kw})
    code = pcbp.pc_construct(N, K, r, poly)
    dec = pcbp.Decoder(code, s, max_iters, dev)
    dec(torch.from_numpy(np.ascontiguousarray(llr)).to(dev))
    torch.cuda.synchronize()
    assert status_of(dec) == 0, f"out-of-range access classes {status_of(dec):#x}"
