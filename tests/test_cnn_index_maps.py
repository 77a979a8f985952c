"""The im2col / layout index maps of the secure CNN against a direct convolution (CPU)."""
import numpy as np

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
