"""ChaCha20 block function (RFC 8439 Sec. 2.3) as the pairwise-seeded PRG (oracle).

Paper, Sec. 2 "Secret sharing": when parties P_j and P_k "pick random values together" they invoke
a PRG with their common seed eta_{j,k}.  The paper names no PRG; reading: the ChaCha20 block
function in counter mode, keyed per party pair, with a 96-bit nonce that names the stream.

Stream layout (shared definition, restated independently in the CUDA path):
  * pair keys: eta_{0,1}, eta_{0,2}, eta_{1,2} = first 32 bytes of ChaCha20(master seed,
    counter 0, nonce words (0x0059454B, pair, 0)) with pair = 1, 2, 3;
  * element i of stream (tag, obj) is the little-endian u64 formed by state words 2w, 2w+1
    (w = i mod 8) of the block with counter floor(i / 8) and nonce words
    (tag, obj mod 2^32, obj >> 32).

Pins (tests/test_oracle_prf.py): the RFC 8439 Sec. 2.3.2 block test vector (tests/golden), and the
`cryptography` package's ChaCha20 keystream for random keys, nonces and counters.
"""
from __future__ import annotations

import numpy as np

_SIGMA = np.array([0x61707865, 0x3320646E, 0x79622D32, 0x6B206574], dtype=np.uint32)

KEY_TAG = 0x0059454B  # "KEY\0" little-endian
PAIR_01, PAIR_02, PAIR_12 = 1, 2, 3


def _rotl(x: np.ndarray, n: int) -> np.ndarray:
    return (x << np.uint32(n)) | (x >> np.uint32(32 - n))


def _quarter(s, a, b, c, d):
    s[a] += s[b]; s[d] ^= s[a]; s[d] = _rotl(s[d], 16)
    s[c] += s[d]; s[b] ^= s[c]; s[b] = _rotl(s[b], 12)
    s[a] += s[b]; s[d] ^= s[a]; s[d] = _rotl(s[d], 8)
    s[c] += s[d]; s[b] ^= s[c]; s[b] = _rotl(s[b], 7)


def chacha20_blocks(key_words, counters, nonce_words) -> np.ndarray:
    """ChaCha20 blocks for a vector of 32-bit counters: returns uint32 array (n, 16)."""
    key_words = np.asarray(key_words, dtype=np.uint32)
    counters = np.asarray(counters, dtype=np.uint64)
    assert key_words.shape == (8,)
    assert np.all(counters < (1 << 32)), "block counter exceeds 32 bits"
    n = counters.shape[0]
    init = np.empty((16, n), dtype=np.uint32)
    init[0:4] = _SIGMA[:, None]
    init[4:12] = key_words[:, None]
    init[12] = counters.astype(np.uint32)
    init[13:16] = np.asarray(nonce_words, dtype=np.uint32)[:, None]
    s = init.copy()
    for _ in range(10):
        _quarter(s, 0, 4, 8, 12); _quarter(s, 1, 5, 9, 13)
        _quarter(s, 2, 6, 10, 14); _quarter(s, 3, 7, 11, 15)
        _quarter(s, 0, 5, 10, 15); _quarter(s, 1, 6, 11, 12)
        _quarter(s, 2, 7, 8, 13); _quarter(s, 3, 4, 9, 14)
    return (s + init).T.copy()


def key_from_bytes(b: bytes) -> np.ndarray:
    assert len(b) == 32
    return np.frombuffer(b, dtype="<u4").astype(np.uint32)


def derive_pair_keys(master_seed: bytes) -> dict:
    """eta_{0,1}, eta_{0,2}, eta_{1,2} from the 32-byte master seed."""
    mk = key_from_bytes(master_seed)
    keys = {}
    for pair in (PAIR_01, PAIR_02, PAIR_12):
        blk = chacha20_blocks(mk, np.array([0], dtype=np.uint64),
                              np.array([KEY_TAG, pair, 0], dtype=np.uint32))[0]
        keys[pair] = blk[:8].copy()
    return keys


def prf_u64(key_words, tag: int, obj: int, start: int, count: int) -> np.ndarray:
    """Elements [start, start+count) of the u64 stream (tag, obj) under ``key_words``."""
    if count == 0:
        return np.zeros(0, dtype=np.uint64)
    assert 0 <= tag < (1 << 32) and 0 <= obj < (1 << 64)
    idx = np.arange(start, start + count, dtype=np.uint64)
    blocks = idx >> np.uint64(3)
    ublk, inv = np.unique(blocks, return_inverse=True)
    nonce = np.array([tag, obj & 0xFFFFFFFF, obj >> 32], dtype=np.uint32)
    words = chacha20_blocks(key_words, ublk, nonce)  # (nb, 16)
    w = (idx & np.uint64(7)).astype(np.int64)
    lo = words[inv, 2 * w].astype(np.uint64)
    hi = words[inv, 2 * w + 1].astype(np.uint64)
    return lo | (hi << np.uint64(32))
