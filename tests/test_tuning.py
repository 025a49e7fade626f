"""The autotune cache (paper_2212_14191_gb300/tuning.py) on the CPU, with the library calls
replaced by a fake binding: a miss runs the autotuner and records its choice under the
(GPU, N, limbs, batch) key, a later process hits the file and sets the stored variants
without timing, stale or inapplicable entries and unreadable files fall back to tuning."""
import json

import pytest

from paper_2212_14191_gb300 import tuning as T


class FakeFhe:
    class FheError(Exception):
        pass

    def __init__(self, count=8, best=(6, 3), bad=()):
        self.count, self.best, self.bad = count, best, set(bad)
        self.tuned = 0
        self.variant = {0: 0, 1: 0}
        self.set_calls = []

    def fhe_ntt_variant_count(self, ctx, logN):
        return self.count

    def fhe_ntt_set_variant(self, ctx, logN, fwd, inv):
        if fwd in self.bad or inv in self.bad:
            raise self.FheError("variant does not apply")
        self.set_calls.append((fwd, inv))
        self.variant = {0: fwd, 1: inv}

    def fhe_ntt_get_variant(self, ctx, logN, inverse):
        return self.variant[inverse]

    def fhe_autotune_ntt(self, ctx, logN, d_ptr, n_limbs, batch, reps=2, stream=0):
        self.tuned += 1
        self.variant = {0: self.best[0], 1: self.best[1]}
        ms = [float(10 + v) for v in range(self.count)]
        return ms, [m + 0.5 for m in ms]


def test_miss_tunes_and_records_then_a_new_process_hits(tmp_path):
    path = str(tmp_path / "tune.json")
    f = FakeFhe()
    got, hit = T.tuned_variants(f, 1, 16, 0, 44, 64, "GB300", T.TuneCache(path))
    assert got == (6, 3) and not hit and f.tuned == 1
    data = json.load(open(path))
    key = T.cache_key("GB300", 16, 44, 64)
    assert data[key]["fwd"] == 6 and data[key]["inv"] == 3 and data[key]["ms"] == {"fwd": 16.0, "inv": 13.5}
    f2 = FakeFhe(best=(0, 0))
    got, hit = T.tuned_variants(f2, 1, 16, 0, 44, 64, "GB300", T.TuneCache(path))
    assert got == (6, 3) and hit and f2.tuned == 0 and f2.set_calls == [(6, 3)]
    # another workload or GPU is another key
    got, hit = T.tuned_variants(f2, 1, 16, 0, 44, 32, "GB300", T.TuneCache(path))
    assert not hit and f2.tuned == 1


@pytest.mark.parametrize("entry", [{"fwd": 9, "inv": 1}, {"fwd": 2, "inv": 5}])
def test_stale_or_inapplicable_entries_tune_again(tmp_path, entry):
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({T.cache_key("GB300", 15, 44, 128): entry}))
    f = FakeFhe(count=8, best=(4, 4), bad=(5,))      # 9 is out of range, 5 does not apply
    got, hit = T.tuned_variants(f, 1, 15, 0, 44, 128, "GB300", T.TuneCache(str(path)))
    assert got == (4, 4) and not hit and f.tuned == 1
    assert json.loads(path.read_text())[T.cache_key("GB300", 15, 44, 128)]["fwd"] == 4


@pytest.mark.parametrize("content", ["not json", "[1, 2]", '{"k": {"fwd": "x", "inv": 1}}'])
def test_unreadable_files_start_empty(tmp_path, content):
    path = tmp_path / "tune.json"
    path.write_text(content)
    assert T.TuneCache(str(path)).entries == {}
    assert T.TuneCache(str(tmp_path / "missing.json")).entries == {}
