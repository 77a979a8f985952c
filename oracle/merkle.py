"""Hash H of Pi_Rec: SHA-256 Merkle root over 1 KiB leaves (oracle; test infrastructure only).

Paper, Sec. 2 "Verifiability of share reconstruction": in Pi_Rec, P1 sends H([r_x]_1) to P2, P2
sends H(m_x) to P0 and H([r_x]_2) to P1; a party aborts when a received value and a received hash
disagree.  The paper does not name H.  Reading: SHA-256 (FIPS 180-4) of each 1024-byte leaf of the
little-endian byte image of the u64 array (the last leaf may be shorter), then a binary tree whose
node is SHA-256(left || right); an odd node at the end of a level is promoted unchanged.  (Any
collision-resistant H serves the check; short leaves let many leaves be hashed in parallel.)  An empty
array hashes to SHA-256 of the empty string.  The array length is public, so no domain prefix is
needed.

Pins (tests/test_oracle_prf.py): FIPS 180-2 "abc" digest; tree shape on hand-built inputs.
"""
from __future__ import annotations

import hashlib

import numpy as np

LEAF_BYTES = 1024


def sha256(b: bytes) -> bytes:
    return hashlib.sha256(b).digest()


def merkle_root_bytes(data: bytes) -> bytes:
    if len(data) == 0:
        return sha256(b"")
    level = [sha256(data[i:i + LEAF_BYTES]) for i in range(0, len(data), LEAF_BYTES)]
    while len(level) > 1:
        nxt = [sha256(level[i] + level[i + 1]) for i in range(0, len(level) - 1, 2)]
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    return level[0]


def hash_u64(arr) -> bytes:
    """H of a u64 array (flattened in C order, little-endian)."""
    a = np.ascontiguousarray(np.asarray(arr, dtype=np.uint64)).astype("<u8", copy=False)
    return merkle_root_bytes(a.tobytes())
