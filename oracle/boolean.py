"""Boolean <.>^1 sharings over Z_2 and their verification ring GF(2^64) = GR(2, 64) (oracle; test
infrastructure only).

Sec. 4.3: Boolean shares are shares over the ring Z_2 (l = 1); AND gates are Pi_Mult over Z_2 and
are verified with Pi_MultVerify over the extension ring of degree d, here GR(2, 64) = GF(2^64)
with the same f = x^64 + x^4 + x^3 + x + 1.  All protocol code of `protocols` and `verify` is
generic in the session's ring, so a BoolSession (l = 1, d = 64) runs the same functions; only the
wire and stream conventions are Boolean:

  - a Boolean stream yields bits: bit i of a (purpose, component, object) stream is bit i mod 64
    of ChaCha20 word floor(i / 64) (64 bits per word, not one per word);
  - a GF(2^64) element drawn from a stream is one whole word (bit c = coefficient of x^c);
  - on the wire and under the Pi_Rec hash, bit arrays are packed the same way (element i of the
    C-order flattening -> bit i mod 64 of word floor(i / 64)); a message of k bits costs
    8 * ceil(k / 64) bytes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .chacha import prf_u64
from .galois import GR
from .shares import LedgerEntry, Session, _COMP_PAIR, tag

U64 = np.uint64


def gf64() -> GR:
    """GR(2, 64) = GF(2^64) with the modulus of GR(2^64, 64)."""
    return GR(ell=1, d=64)


def pack_bits(bits) -> np.ndarray:
    """0/1 array (any shape, C order) -> u64 words, element i at bit i mod 64 of word i // 64."""
    b = np.asarray(bits, dtype=U64).reshape(-1) & U64(1)
    nw = (b.size + 63) // 64
    pad = np.zeros(nw * 64, dtype=U64)
    pad[: b.size] = b
    sh = np.arange(64, dtype=U64)
    return np.bitwise_or.reduce(pad.reshape(nw, 64) << sh, axis=1).astype(U64) if nw else pad[:0]


def unpack_bits(words, count: int) -> np.ndarray:
    """Inverse of pack_bits for the first `count` elements."""
    w = np.asarray(words, dtype=U64).reshape(-1)
    sh = np.arange(64, dtype=U64)
    return ((w[:, None] >> sh) & U64(1)).reshape(-1)[:count].astype(U64)


@dataclass
class BoolSession(Session):
    """A session over Z_2 whose verification ring is GF(2^64)."""
    gr: GR = field(default_factory=gf64)

    def prf(self, comp: int, purpose: int, obj: int, count: int, start: int = 0) -> np.ndarray:
        key = self.keys[_COMP_PAIR[comp]]
        if count <= 0:
            return np.zeros(0, dtype=U64)
        w0 = start // 64
        w1 = (start + count - 1) // 64
        words = prf_u64(key, tag(purpose, comp), obj, w0, w1 - w0 + 1)
        bits = unpack_bits(words, (w1 - w0 + 1) * 64)
        return bits[start - 64 * w0: start - 64 * w0 + count]

    def prf_gr(self, comp: int, purpose: int, obj: int, n: int = None) -> np.ndarray:
        """GF(2^64) elements: element i is stream word i, coefficient c its bit c."""
        key = self.keys[_COMP_PAIR[comp]]
        k = 1 if n is None else n
        words = prf_u64(key, tag(purpose, comp), obj, 0, k)
        el = unpack_bits(words, 64 * k).reshape(k, 64)
        return el[0] if n is None else el

    def wire(self, arr) -> np.ndarray:
        return pack_bits(arr)

    def send(self, src: int, dst: int, phase: str, proto: str, arr, site: str = None,
             nbytes: int = None) -> np.ndarray:
        arr = np.array(arr, dtype=U64, copy=True)
        if nbytes is None:
            nbytes = 8 * ((arr.size + 63) // 64)
        return super().send(src, dst, phase, proto, arr, site=site, nbytes=nbytes)


def gf_to_words(el) -> np.ndarray:
    """GF(2^64) elements as (..., 64) coefficient bits -> u64 words (bit c = coefficient c)."""
    e = np.asarray(el, dtype=U64)
    sh = np.arange(64, dtype=U64)
    return np.bitwise_or.reduce((e & U64(1)) << sh, axis=-1).astype(U64)


def words_to_gf(words) -> np.ndarray:
    w = np.asarray(words, dtype=U64)
    sh = np.arange(64, dtype=U64)
    return (w[..., None] >> sh) & U64(1)


__all__ = ["BoolSession", "gf64", "pack_bits", "unpack_bits", "gf_to_words", "words_to_gf",
           "LedgerEntry"]
