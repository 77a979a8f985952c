"""Config C2 on the GPU: secure 784-128-128-10 MLP inference, batch 128, 13 fractional bits,
weights N(0, 0.05^2), inputs U[0, 1).  Every layer's products, truncation pairs and ReLU are
verified; the opened logits stay within 2^-8 of a float64 model evaluated on the decoded
fixed-point inputs and weights (the protocol's error bound; reading A10)."""
import hashlib

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


@pytest.mark.parametrize("path", [1, 0])
def test_secure_mlp_logits_within_bound(mpc, path):
    from paper_2411_09287_gb300 import secure_mlp as SM
    from paper_2411_09287_gb300 import workloads
    k = 13
    sizes = [784, 128, 128, 10]
    weights = SM.mlp_weights(sizes, "C2-weights")
    x = workloads.rng("C2-inputs").uniform(0.0, 1.0, (128, 784))
    ctx = mpc.Context(hashlib.sha256(b"mpc3-config-C2").digest(), gemm_path=path)
    got = SM.secure_forward(ctx, x, weights, k)
    ref = SM.fp64_forward(SM.quantized(x, k), [SM.quantized(w, k) for w in weights])
    err = np.abs(got - ref)
    assert err.max() <= 2.0 ** -8, err.max()
    # the secure network computes the same classification as the float64 model
    assert np.mean(np.argmax(got, axis=1) == np.argmax(ref, axis=1)) > 0.95


@pytest.mark.parametrize("path", [1])
def test_secure_cnn_net_a_within_bound(mpc, path):
    """Config C4, Net A (reading A17): conv 5x5x16, pool, conv 5x5x16, pool, FC 256-100-10 over
    im2col share GEMMs, batch 8; He-normal weights, inputs U[0, 1)."""
    from paper_2411_09287_gb300 import secure_cnn as SC
    from paper_2411_09287_gb300 import secure_mlp as SM
    from paper_2411_09287_gb300 import workloads
    k = 13
    p = SC.net_a_params("C4-netA-weights")
    x = workloads.rng("C4-netA-inputs").uniform(0.0, 1.0, (8, 1, 28, 28))
    ctx = mpc.Context(hashlib.sha256(b"mpc3-config-C4").digest(), gemm_path=path)
    got = SC.net_a_secure(ctx, x, p, k)
    q = lambda a: SM.quantized(a, k)
    ref = SC.net_a_fp64(q(x), {n: q(w) for n, w in p.items()})
    err = np.abs(got - ref)
    assert err.max() <= 2.0 ** -8, err.max()


def test_secure_cnn_net_b_within_bound(mpc):
    """Config C4, Net B (reading A17): five 3x3 pad-1 convs with pools after the second, fourth
    and fifth, FC 4096-512-10; one image, He-normal weights, inputs U[0, 1)."""
    from paper_2411_09287_gb300 import secure_cnn as SC
    from paper_2411_09287_gb300 import secure_mlp as SM
    from paper_2411_09287_gb300 import workloads
    k = 13
    p = SC.net_b_params("C4-netB-weights")
    x = workloads.rng("C4-netB-inputs").uniform(0.0, 1.0, (1, 3, 32, 32))
    ctx = mpc.Context(hashlib.sha256(b"mpc3-config-C4-netB").digest())
    got = SC.net_b_secure(ctx, x, p, k)
    q = lambda a: SM.quantized(a, k)
    ref = SC.net_b_fp64(q(x), {n: q(w) for n, w in p.items()})
    assert np.max(np.abs(got - ref)) <= 2.0 ** -8
