"""Named parameter sets of the workloads this library is measured and tested on, restating the
paper's parameter tables (Table V's default N = 2^16 and L = 44; the HMULT key-switching
configuration with 24 ciphertext limbs, 8 special primes and slices of 8; the default batch of
Sec. VI-E, the batch-size study; the HEAX comparison sets of Table VIII with this library's 30-bit primes). The
benchmark reads its sizes from here; a user can take the same sets.

Every modulus set is the library's prime sequence (fhe_gen_primes / oracle.params): 30-bit
primes q = 1 mod 2^17 in descending order, the special primes taken first.
"""
from dataclasses import dataclass


@dataclass(frozen=True)
class NttWorkload:
    """Forward + inverse transforms of `batch` polynomials over each of `limbs` moduli."""
    logN: int
    limbs: int
    batch: int


@dataclass(frozen=True)
class HmultWorkload:
    """HMULT + relinearisation + rescale of `batch` ciphertext pairs with `limbs` ciphertext
    limbs, `special` special primes and key-switching slices of `alpha` limbs."""
    logN: int
    limbs: int
    special: int
    alpha: int
    batch: int

    @property
    def dnum(self):
        return -(-self.limbs // self.alpha)


@dataclass(frozen=True)
class MixedBatch:
    """`ops` operations drawn uniformly from NTT / INTT / HMULT, ring degrees `logNs` and
    `limb_range` (inclusive) ciphertext limbs, one polynomial or pair each."""
    ops: int
    logNs: tuple
    limb_range: tuple
    special: int
    alpha: int


@dataclass(frozen=True)
class ServingStream:
    """Poisson arrivals at `rate_per_s` of HMULT / RESCALE / KEYSWITCH requests over ring
    degrees `logNs` and `limb_range` (inclusive) limbs, admitted under `budget_bytes`."""
    rate_per_s: float
    logNs: tuple
    limb_range: tuple
    budget_bytes: int
    streams: int
    max_batch: int


@dataclass(frozen=True)
class HeaxSet:
    """A HEAX comparison set: ring degree 2^logN, L ciphertext limbs and K special primes
    (log PQ / 30 rounded up, P > Q, one key-switching slice)."""
    name: str
    logN: int
    L: int
    K: int


NTT_SMALL = NttWorkload(logN=12, limbs=1, batch=16)            # the small parity case
NTT_FULL = NttWorkload(logN=16, limbs=44, batch=64)            # the benchmarked step, 704 MiB
HMULT_FULL = HmultWorkload(logN=16, limbs=24, special=8, alpha=8, batch=128)
MIXED_BATCH = MixedBatch(ops=1000, logNs=(14, 15, 16), limb_range=(3, 44), special=8, alpha=8)
SERVING = ServingStream(rate_per_s=50000.0, logNs=(15, 16), limb_range=(3, 24), budget_bytes=24 << 30,
                        streams=4, max_batch=32)
HEAX_SETS = (HeaxSet("Set_A", 12, 2, 2), HeaxSet("Set_B", 13, 4, 4), HeaxSet("Set_C", 14, 7, 8))
HEAX_BATCH = 1024
# batch sizes of the sets' batch-size sensitivity (Sec. VI-E: 32 to 1024 ciphertexts per call)
HEAX_BATCH_SWEEP = (32, 64, 128, 256, 512, 1024)
