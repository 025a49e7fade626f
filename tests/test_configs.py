"""The named parameter sets (paper_2212_14191_gb300/configs.py) on the CPU: the sizes the
benchmark and the documentation quote, the benchmark reading them, and the key-switching
condition P > Q_j of every set with the library's primes (special primes first)."""
import math

import bench
from oracle import params as P
from paper_2212_14191_gb300 import configs as CFG


def test_workload_sizes():
    w = CFG.NTT_FULL
    assert (w.logN, w.limbs, w.batch) == (16, 44, 64)
    assert w.limbs * w.batch * (1 << w.logN) * 4 == 704 << 20          # 704 MiB, above the 129 MB L2
    h = CFG.HMULT_FULL
    assert (h.logN, h.limbs, h.special, h.alpha, h.batch, h.dnum) == (16, 24, 8, 8, 128, 3)
    assert CFG.MIXED_BATCH.ops == 1000 and CFG.MIXED_BATCH.logNs == (14, 15, 16)
    assert CFG.SERVING.rate_per_s == 50000.0 and CFG.SERVING.limb_range == (3, 24)


def test_bench_reads_the_sets():
    assert (bench.LOGN, bench.NTT_LIMBS, bench.NTT_BATCH) == (CFG.NTT_FULL.logN, CFG.NTT_FULL.limbs,
                                                             CFG.NTT_FULL.batch)
    assert (bench.HM_LIMBS, bench.HM_K, bench.HM_ALPHA, bench.HM_BATCH) == (
        CFG.HMULT_FULL.limbs, CFG.HMULT_FULL.special, CFG.HMULT_FULL.alpha, CFG.HMULT_FULL.batch)
    assert bench.HEAX_SETS == tuple((s.name, s.logN, s.L, s.K) for s in CFG.HEAX_SETS)
    # the batch-size study spans 32 to 1024 ciphertexts per call and ends at the main batch
    assert bench.HEAX_BATCH_SWEEP == CFG.HEAX_BATCH_SWEEP
    assert CFG.HEAX_BATCH_SWEEP[0] == 32 and CFG.HEAX_BATCH_SWEEP[-1] == CFG.HEAX_BATCH
    assert list(CFG.HEAX_BATCH_SWEEP) == sorted(set(CFG.HEAX_BATCH_SWEEP))


def test_special_primes_exceed_every_slice():
    allp = P.ntt_primes(60)
    for s in CFG.HEAX_SETS:                                   # one slice: P > Q
        ps, qs = allp[:s.K], allp[s.K:s.K + s.L]
        assert math.prod(ps) > math.prod(qs), s.name
    h = CFG.HMULT_FULL
    ps, qs = allp[:h.special], allp[h.special:h.special + h.limbs]
    for j in range(h.dnum):
        assert math.prod(ps) > math.prod(qs[j * h.alpha:(j + 1) * h.alpha])
