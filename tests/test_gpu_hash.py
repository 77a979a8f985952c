"""H of Pi_Rec on the GPU (mpc_hash_u64) against the oracle's SHA-256 Merkle root, byte for byte:
empty and sub-leaf inputs, exact leaf and 64-leaf CTA boundaries, ragged last leaves and ragged
last CTAs, and a message of 2^21 + 5 words (2049 CTAs' subtrees, 12 tree levels above them)."""
import hashlib

import numpy as np
import pytest

from oracle.merkle import LEAF_BYTES, hash_u64
from paper_2411_09287_gb300 import workloads

pytestmark = pytest.mark.gpu

LEAF_WORDS = LEAF_BYTES // 8


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_09287_gb300 import mpc as M
    return M, M.Context(hashlib.sha256(b"merkle-hash").digest())


@pytest.mark.parametrize("n", [0, 1, 7, LEAF_WORDS - 1, LEAF_WORDS, LEAF_WORDS + 1,
                               64 * LEAF_WORDS - 1, 64 * LEAF_WORDS, 64 * LEAF_WORDS + 1,
                               3 * 64 * LEAF_WORDS + 555, 65 * 64 * LEAF_WORDS + 3,
                               (1 << 21) + 5])
def test_merkle_root_matches_oracle(ctx, n):
    import torch
    M, c = ctx
    x = workloads.rng(f"merkle-{n}").integers(0, 2 ** 64, n, dtype=np.uint64, endpoint=False)
    d = torch.from_numpy(x.view(np.int64)).to("cuda")
    assert c.hash_u64(d) == hash_u64(x)
