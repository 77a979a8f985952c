"""The im2col / layout index maps of the secure CNN against a direct convolution (CPU)."""
import numpy as np
import pytest

from paper_2411_09287_gb300 import secure_cnn as SC


def test_im2col_conv_matches_direct_convolution():
    g = np.random.default_rng(5)
    x = g.normal(size=(2, 3, 7, 6))
    w = g.normal(size=(4, 3, 3, 2))
    ref = np.zeros((2, 4, 5, 5))
    for b in range(2):
        for o in range(4):
            for i in range(5):
                for j in range(5):
                    ref[b, o, i, j] = np.sum(x[b, :, i:i + 3, j:j + 2] * w[o])
    assert np.allclose(SC._conv_fp64(x, w), ref)


def test_rows_to_nchw_is_the_transpose():
    B, Co, Ho, Wo = 2, 3, 4, 5
    z = np.arange(B * Ho * Wo * Co)
    got = z[SC.rows_to_nchw_index(B, Co, Ho, Wo)].reshape(B, Co, Ho, Wo)
    assert np.array_equal(got, z.reshape(B, Ho, Wo, Co).transpose(0, 3, 1, 2))


def test_padded_conv_matches_direct_convolution():
    g = np.random.default_rng(6)
    x = g.normal(size=(2, 3, 5, 4))
    w = g.normal(size=(2, 3, 3, 3))
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    ref = np.zeros((2, 2, 5, 4))
    for b in range(2):
        for o in range(2):
            for i in range(5):
                for j in range(4):
                    ref[b, o, i, j] = np.sum(xp[b, :, i:i + 3, j:j + 3] * w[o])
    assert np.allclose(SC._conv_fp64(x, w, pad=1), ref)


def test_net_b_geometry_reaches_the_4096_flatten():
    p = SC.net_b_params("C4-netB-weights")
    assert p["c5"].shape == (256, 128, 3, 3) and p["f1"].shape == (4096, 512)
    x = np.random.default_rng(7).uniform(0, 1, (2, 3, 32, 32))
    assert SC.net_b_fp64(x, p).shape == (2, 10)


@pytest.mark.parametrize("H,W", [(24, 24), (32, 32), (8, 8), (2, 2)])
@pytest.mark.parametrize("budget", [SC.NL_CHUNK, 1000, 1])
def test_pool_chunks_are_the_most_whole_planes_within_the_budget(H, W, budget):
    """A max-pool call takes whole channel planes, 3 H W / 4 comparisons each (three per 2x2
    window): as many as fit in the comparison budget, at least one, at most all."""
    for planes in (1, 7, 1024, 16384):
        step = SC.pool_planes(budget, H, W, planes)
        assert 1 <= step <= planes
        assert step == 1 or 3 * H * W * step <= 4 * budget
        assert step == planes or 3 * H * W * (step + 1) > 4 * budget
