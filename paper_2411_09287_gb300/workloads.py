"""Seeded synthetic inputs shaped like the paper's workloads (no protocol arithmetic here).

Both the CUDA path and the oracle draw their plaintext inputs from these generators, each side
then encodes and shares them with its own code.  Seeds: numpy PCG64 seeded from
SHA-256("mpc3-config-<name>"); the protocol's own randomness comes from the pairwise PRG, keyed by
``master_seed(name)``.

* ``plain_small``: Pi_Inner of X[64 x 128] by W[128 x 64] and Pi_Mult of two 4096-vectors, entries
  uniform in [-4, 4) (real values; encode with 13 fractional bits).
* ``gemm_square(n)`` / ``gemm_shape(M, N, K)``: uniform 64-bit words for the secure GEMM sweep.
"""
from __future__ import annotations

import hashlib

import numpy as np


def master_seed(name: str) -> bytes:
    return hashlib.sha256(f"mpc3-config-{name}".encode()).digest()


def rng(name: str) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int.from_bytes(master_seed(name)[:8], "little")))


def plain_small():
    g = rng("C1")
    X = g.uniform(-4.0, 4.0, (64, 128))
    W = g.uniform(-4.0, 4.0, (128, 64))
    a = g.uniform(-4.0, 4.0, 4096)
    b = g.uniform(-4.0, 4.0, 4096)
    return X, W, a, b


def gemm_shape(M: int, N: int, K: int, name: str = None):
    g = rng(name or f"C3-{M}x{N}x{K}")
    X = g.integers(0, 2**64, (M, K), dtype=np.uint64)
    W = g.integers(0, 2**64, (K, N), dtype=np.uint64)
    return X, W


def gemm_square(n: int):
    return gemm_shape(n, n, n, f"C3-{n}")


def uniform_words(shape, name: str):
    return rng(name).integers(0, 2**64, shape, dtype=np.uint64)
