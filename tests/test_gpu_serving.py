"""Serving (row a9 / config C5 pattern): requests of uneven batch size arriving over time are
admitted by a device-memory budget, packed into shared secure forward passes and run on two
concurrent contexts; every request's logits are within 2^-8 of the float64 model and within
2^-7 of the same request run alone."""
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


def test_continuous_batching_results_match_alone_runs(mpc):
    import hashlib
    from paper_2411_09287_gb300 import serving as S
    model = S.Model("mlp")
    reqs = S.poisson_requests(model, 12, 400.0, 16, "serving-test")
    srv = S.Server(model, n_workers=2, max_batch=32, mem_budget_bytes=8e9)
    out = srv.serve(reqs)
    st = S.Server.stats(out)
    assert st["requests"] == 12 and st["images_per_s"] > 0 and st["p99_ms"] >= st["p50_ms"]
    ctx = mpc.Context(hashlib.sha256(b"serving-alone").digest())
    for r in out:
        ref = model.fp64(r.x)
        assert np.max(np.abs(r.logits - ref)) <= 2.0 ** -8
        alone = model.secure(ctx, r.x, 10_000 + 1000 * r.rid)
        assert np.max(np.abs(r.logits - alone)) <= 2.0 ** -7
