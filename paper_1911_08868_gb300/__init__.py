"""GB300-native partially permuted multi-trellis BP decoding of polar codes.

Implements the decoder of Ranasinghe, Rajatheva and Latva-aho, "Partially
Permuted Multi-Trellis Belief Propagation for Polar Codes" (arXiv 1911.08868)
as hand-written sm_103a CUDA behind the C ABI of ``include/pcbp.h``.

    from paper_1911_08868_gb300 import pcbp      # ctypes binding of libpcbp.so
    from paper_1911_08868_gb300 import inputs    # seeded BPSK/AWGN workloads

Importing ``pcbp`` loads ``libpcbp.so`` and raises if it has not been built
(``python -m paper_1911_08868_gb300._build``); there is no CPU fallback.
"""
