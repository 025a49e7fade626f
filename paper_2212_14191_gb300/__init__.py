"""GB300-native batched negacyclic NTT and CKKS HMULT (TensorFHE, arXiv 2212.14191).

The compute path is the C-ABI library `libfhe.so` (hand-written CUDA for
sm_103a, built from csrc/); `fhe` is its thin ctypes binding.
"""
