"""Pins for the oracle's PRG (ChaCha20) and hash H (SHA-256 Merkle) -- no GPU."""
import hashlib
import os

import numpy as np
import pytest

from oracle.chacha import chacha20_blocks, derive_pair_keys, key_from_bytes, prf_u64
from oracle.merkle import LEAF_BYTES, hash_u64, merkle_root_bytes


def test_chacha20_rfc8439_vector(golden):
    g = golden("chacha20_rfc8439_sec2_3_2.txt")
    key = key_from_bytes(bytes.fromhex(g["key"]))
    nonce = np.frombuffer(bytes.fromhex(g["nonce"]), dtype="<u4")
    blk = chacha20_blocks(key, np.array([int(g["counter"])], dtype=np.uint64), nonce)[0]
    assert blk.astype("<u4").tobytes().hex() == g["block"]


def test_prf_matches_cryptography_keystream():
    algorithms = pytest.importorskip("cryptography.hazmat.primitives.ciphers").algorithms
    Cipher = pytest.importorskip("cryptography.hazmat.primitives.ciphers").Cipher
    rng = np.random.default_rng(7)
    for _ in range(6):
        key = rng.bytes(32)
        tag = int(rng.integers(0, 2**32))
        obj = int(rng.integers(0, 2**63))
        start_block = int(rng.integers(0, 2**20))
        nblocks = int(rng.integers(1, 5))
        words = prf_u64(key_from_bytes(key), tag, obj, start_block * 8, nblocks * 8)
        nonce = tag.to_bytes(4, "little") + (obj & 0xFFFFFFFF).to_bytes(4, "little") + \
            (obj >> 32).to_bytes(4, "little")
        enc = Cipher(algorithms.ChaCha20(key, start_block.to_bytes(4, "little") + nonce),
                     mode=None).encryptor()
        ks = enc.update(bytes(64 * nblocks))
        assert words.astype("<u8").tobytes() == ks


def test_prf_unaligned_ranges_and_pair_keys():
    key = key_from_bytes(bytes(range(32)))
    full = prf_u64(key, 5, 9, 0, 40)
    assert np.array_equal(prf_u64(key, 5, 9, 3, 17), full[3:20])
    keys = derive_pair_keys(hashlib.sha256(b"s").digest())
    assert len({bytes(v) for v in keys.values()}) == 3


def test_sha256_fips_vector(golden):
    g = golden("sha256_fips180_abc.txt")
    assert merkle_root_bytes(bytes.fromhex(g["message"])).hex() == g["digest"]


def test_merkle_shapes():
    h = lambda b: hashlib.sha256(b).digest()
    a = os.urandom(LEAF_BYTES)
    b = os.urandom(LEAF_BYTES)
    c = os.urandom(100)
    assert merkle_root_bytes(b"") == h(b"")
    assert merkle_root_bytes(a) == h(a)
    assert merkle_root_bytes(a + b) == h(h(a) + h(b))
    assert merkle_root_bytes(a + b + c) == h(h(h(a) + h(b)) + h(c))   # odd node promoted
    arr = np.arange(10, dtype=np.uint64)
    assert hash_u64(arr) == h(arr.astype("<u8").tobytes())
    # five leaves: promotions on two levels
    ls = [os.urandom(LEAF_BYTES) for _ in range(4)] + [c]
    hh = [h(x) for x in ls]
    assert merkle_root_bytes(b"".join(ls)) == h(h(h(hh[0] + hh[1]) + h(hh[2] + hh[3])) + hh[4])
