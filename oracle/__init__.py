"""CPU oracle for the TensorFHE hot path (arXiv 2212.14191).

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import anything from this package. The GPU
library shares no code with it: it computes its own primes, roots and tables,
and the oracle never imports the GPU package.

Modules
  params  -- NTT-friendly primes and primitive 2N-th roots (Sec. II-A)
  ntt     -- ctypes wrapper around ntt_oracle.c (Eq. (4) and its inverse)
  ckks    -- full-RNS CKKS: basis conversion, key switching, HMULT, rescale,
             encode/decode and encryption (Sec. II-B, Sec. IV-A)
"""
