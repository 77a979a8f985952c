"""Serving (row a9 / config C5 pattern): requests of uneven batch size arriving over time are
admitted by a device-memory budget, packed into shared secure forward passes and run on two
concurrent contexts of the same three parties, with the weights shared once per worker.  Every
request's logits are within 2^-8 of the float64 model and bit-identical to the same request run
alone (its truncation bits are keyed by request, layer and row)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_09287_gb300 import mpc as M
    return M


@pytest.mark.parametrize("kind,nreq,maxb,budget", [("mlp", 12, 16, 8e9), ("neta", 5, 3, 64e9)])
def test_packed_requests_are_bit_identical_to_alone_runs(mpc, kind, nreq, maxb, budget):
    from paper_2411_09287_gb300 import serving as S
    model = S.Model(kind)
    reqs = S.poisson_requests(model, nreq, 400.0, maxb, f"serving-test-{kind}")
    srv = S.Server(model, n_workers=2, max_batch=2 * maxb, mem_budget_bytes=budget)
    out = srv.serve(reqs)
    st = S.Server.stats(out)
    assert st["requests"] == nreq and st["images_per_s"] > 0 and st["p99_ms"] >= st["p50_ms"]
    packed = sum(1 for r in out if r.x.shape[0] < 2 * maxb) > 0
    assert packed
    ctx = mpc.Context(S.Server.SEED)
    shared = model.share(ctx, 1 << 40)
    for r in out:
        assert r.error is None
        assert np.max(np.abs(r.logits - model.fp64(r.x))) <= 2.0 ** -8
        alone = model.secure(ctx, r.x, (1 << 41) + 1000 * r.rid, shared, [(r.rid, r.x.shape[0])])
        assert np.array_equal(r.logits, alone), f"request {r.rid}"
