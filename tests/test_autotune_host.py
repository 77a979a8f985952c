"""Host logic of the autotuner on CPU, with a stand-in for the library: coordinate descent keeps
the fastest candidate of every knob group given the best of the earlier groups, a candidate that
changes the verification transcript is refused, and picks are cached per key."""
import numpy as np
import pytest

from paper_2411_09287_gb300 import autotune as AT


class _Ctx:
    def __init__(self, tuning):
        self.tuning = tuning

    def close(self):
        pass


def _cost(t):
    # separable costs with a known optimum: split 16, gram 152, row split 384
    return (10.0 + {8: 3.0, 4: 5.0, 16: 1.0}[t.get("gemm_split_min", 8)]
            + {76: 2.0, 152: 0.5, 38: 4.0}[t.get("gram_split", 76)]
            + {0: 1.0, 384: 0.2, 128: 2.0}[t.get("row_split", 0)])


def _clock(ctx, fn):
    return _cost(ctx.tuning), fn()


SPACE = [("split", [dict(gemm_split_min=v) for v in (8, 4, 16)]),
         ("gram", [dict(gram_split=v) for v in (76, 152, 38)]),
         ("rowsplit", [dict(row_split=v) for v in (0, 384, 128)])]


def test_coordinate_descent_finds_the_separable_optimum():
    rec = AT.autotune(_Ctx, lambda ctx: np.arange(5), SPACE, clock=_clock)
    assert rec["picks"] == dict(gemm_split_min=16, gram_split=152, row_split=384)
    assert len(rec["trials"]) == 9
    # later groups were timed with the earlier groups' picks in force
    gram = [tr for tr in rec["trials"] if tr["group"] == "gram"]
    assert min(g["ms"] for g in gram) == pytest.approx(_cost(dict(gemm_split_min=16, gram_split=152)))


def test_a_candidate_that_changes_the_transcript_is_refused():
    def step(ctx):
        bad = ctx.tuning.get("gram_split") == 38
        return np.arange(5) + (1 if bad else 0)
    with pytest.raises(AT.TranscriptMismatch):
        AT.autotune(_Ctx, step, SPACE, clock=_clock)


def test_row_split_candidates_are_odd_multiples_of_128():
    for E in (1 << 10, 1 << 20, 1 << 24, 12345):
        c = AT._row_split_candidates(E)
        assert c[0] == 0
        assert all(v % 128 == 0 and (v // 128) % 2 == 1 and v <= E for v in c[1:])


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setenv("MPC3_AUTOTUNE_CACHE", str(tmp_path / "at.json"))
    key = AT._key("GB300", 8, 8, 8, 13, 1)
    assert AT.load_cached(key) is None
    AT.store_cached(key, {"picks": {"gram_split": 152}})
    assert AT.load_cached(key) == {"picks": {"gram_split": 152}}
    AT.store_cached(AT._key("GB300", 16, 8, 8, 13, 1), {"picks": {}})
    assert AT.load_cached(key) == {"picks": {"gram_split": 152}}
