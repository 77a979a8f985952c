"""Host logic of the continuous-batching server on CPU: requests are admitted in arrival order as
long as their images fit the limit, and a request that could never fit is refused up front
instead of stalling the server."""
import numpy as np
import pytest

from paper_2411_09287_gb300 import serving as S


def _reqs(sizes):
    return [S.Request(i, 0.01 * i, np.zeros((b, 4))) for i, b in enumerate(sizes)]


def test_pack_admits_the_longest_fitting_prefix_in_order():
    pending = _reqs([3, 5, 2, 1])
    pack, n = S.pack_requests(pending, 8)
    assert [r.rid for r in pack] == [0, 1] and n == 8
    assert [r.rid for r in pending] == [2, 3]
    pack, n = S.pack_requests(pending, 8)
    assert [r.rid for r in pack] == [2, 3] and n == 3 and not pending


def test_pack_keeps_order_when_the_head_does_not_fit():
    pending = _reqs([6, 1])
    pack, n = S.pack_requests(pending, 5)
    assert pack == [] and n == 0 and [r.rid for r in pending] == [0, 1]


def test_pack_never_exceeds_the_limit():
    rng = np.random.default_rng(5)
    pending = _reqs(list(rng.integers(1, 9, 200)))
    total = 0
    while pending:
        pack, n = S.pack_requests(pending, 16)
        assert pack and n <= 16 and n == sum(r.x.shape[0] for r in pack)
        total += n
    assert total == sum(r.x.shape[0] for r in _reqs(list(np.random.default_rng(5).integers(1, 9, 200))))


@pytest.mark.parametrize("max_batch,max_in_flight,ok", [(32, 1000, True), (4, 1000, False),
                                                        (32, 4, False)])
def test_requests_that_can_never_fit_are_refused(max_batch, max_in_flight, ok):
    reqs = _reqs([3, 5, 2])
    if ok:
        S.check_admissible(reqs, max_batch, max_in_flight)
    else:
        with pytest.raises(ValueError):
            S.check_admissible(reqs, max_batch, max_in_flight)


class _StubModel:
    """secure() fails on the chosen call; bytes_per_image is a constant."""

    def __init__(self, fail_on: int):
        self.fail_on, self.calls = fail_on, 0

    def bytes_per_image(self, ctx, b):
        return 1.0

    def share(self, ctx, call_base):
        return "resident weights"

    def secure(self, ctx, x, call_base, shared=None, segments=None):
        assert shared == "resident weights" and sum(b for _, b in segments) == x.shape[0]
        self.calls += 1
        if self.calls == self.fail_on:
            raise RuntimeError("protocol aborted")
        return np.full((x.shape[0], 10), float(call_base))


@pytest.mark.parametrize("fail_on", [None, 1, 3])
def test_a_failed_pass_is_reported_and_never_hangs_the_server(fail_on):
    model = _StubModel(fail_on or 10**9)
    srv = S.Server(model, n_workers=2, max_batch=4, mem_budget_bytes=64,
                   make_context=lambda wid: (f"stub context {wid}", None))
    reqs = _reqs([1, 2, 3, 1, 2, 4, 1])
    if fail_on is None:
        out = srv.serve(reqs)
        assert all(r.logits is not None and r.error is None for r in out)
    else:
        with pytest.raises(RuntimeError, match="protocol aborted"):
            srv.serve(reqs)
        assert any(r.error is not None for r in reqs)
    assert srv.in_flight == 0
    assert all(not w.is_alive() for w in srv.workers)
