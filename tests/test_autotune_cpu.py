"""CPU checks of the autotuner's host side: the workload key, the JSON cache and its use by `tuned`
(a fake target stands in for a graph), and the C-ABI's argument checks (no GPU needed)."""
import ctypes

import pytest


class FakeTarget:
    """Records what `tuned` asks of a graph: set_options on a cache hit, autotune on a miss."""

    def __init__(self, mf, ms=12.5):
        self.mf = mf
        self.ms = ms
        self.set_calls = []
        self.tune_calls = 0

    def set_options(self, o):
        self.set_calls.append(self.mf.options_to_dict(o))

    def autotune(self, reps=3, sweeps=1, time_budget_ms=0.0):
        self.tune_calls += 1
        return self.mf.default_options(bin_warp=128, gr_time_ratio=4.0), self.ms


def test_workload_key_rounds_sizes_to_powers_of_two():
    from paper_1507_01926_gb300 import autotune as A

    assert A.workload_key("grid3d", 8388610, 50331648) == A.workload_key("grid3d", 9000000, 40000000)
    assert A.workload_key("grid3d", 1000, 5000) != A.workload_key("grid3d", 5000, 5000)
    assert A.workload_key("layered", 1000, 5000, 64) != A.workload_key("layered", 1000, 5000, 128)
    assert A.workload_key("a", 10, 10) != A.workload_key("b", 10, 10)


def test_options_dict_round_trip(built):
    from paper_1507_01926_gb300 import mf

    o = mf.default_options(bin_warp=256, gr_freq=1.0, block_threads=128, blocks_per_sm=4)
    d = mf.options_to_dict(o)
    assert d["bin_warp"] == 256 and d["gr_freq"] == 1.0
    assert mf.options_to_dict(mf.options_from_dict(d)) == d
    with pytest.raises(KeyError):
        mf.options_from_dict({"no_such_field": 1})


def test_cache_miss_tunes_and_stores_then_hit_applies(built, tmp_path):
    from paper_1507_01926_gb300 import autotune as A
    from paper_1507_01926_gb300 import mf

    path = str(tmp_path / "tune.json")
    key = A.workload_key("layered", 84000, 420000, 64)
    t1 = FakeTarget(mf)
    o1, ms1, hit1 = A.tuned(t1, key, path=path)
    assert (hit1, t1.tune_calls, ms1) == (False, 1, 12.5)
    assert A.lookup(key, A.device_name(0), path) is not None
    t2 = FakeTarget(mf)
    o2, ms2, hit2 = A.tuned(t2, key, path=path)
    assert hit2 and t2.tune_calls == 0 and ms2 == 12.5
    assert t2.set_calls == [mf.options_to_dict(o2)]
    assert mf.options_to_dict(o2) == mf.options_to_dict(o1)
    # another key or retune=True tunes again
    t3 = FakeTarget(mf, ms=3.0)
    _, ms3, hit3 = A.tuned(t3, key, path=path, retune=True)
    assert not hit3 and t3.tune_calls == 1 and A.lookup(key, A.device_name(0), path)[1] == 3.0
    # a corrupt cache file reads as empty
    open(path, "w").write("{not json")
    assert A.load_cache(path) == {}


def test_tuning_entry_points_reject_null_arguments(built):
    from paper_1507_01926_gb300 import mf

    L = mf.lib()
    o = mf.default_options()
    assert L.mf_set_options(None, ctypes.byref(o)) == -1
    assert L.mf_autotune(None, None, None, None) == -1
    assert L.mf_batch_set_options(None, ctypes.byref(o)) == -1
    assert L.mf_batch_autotune(None, None, None, None) == -1
    assert b"null" in L.mf_last_error()


def test_packaged_table_is_a_fallback_of_valid_options(built, tmp_path):
    from paper_1507_01926_gb300 import autotune as A
    from paper_1507_01926_gb300 import mf

    table = A.load_cache(A.PACKAGED)
    assert "NVIDIA GB300" in table and len(table["NVIDIA GB300"]) == 3
    for key, e in table["NVIDIA GB300"].items():
        o = mf.options_from_dict(e["options"])  # every field is an mf_options field
        assert o.block_threads % 32 == 0 and o.bin_warp >= o.bin_thread and e["ms"] > 0
        empty = str(tmp_path / "none.json")
        hit = A.lookup(key, "NVIDIA GB300", empty)
        assert hit is not None and mf.options_to_dict(hit[0]) == mf.options_to_dict(o)
        assert A.lookup(key, "NVIDIA GB300", empty, packaged=False) is None
        assert A.lookup(key, "some other device", empty) is None
    assert A.workload_key("grid3d", 8388610, 50331648) in table["NVIDIA GB300"]
