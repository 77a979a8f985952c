"""Galois ring GR(2^l, d) = Z_2^l[x] / f(x) (oracle; test infrastructure only).

Paper: Sec. 2 "Notation" defines the sharings [.]^{l[x]}, <.>^{l[x]} over Z_2^l[x]/f(x) with f a
degree-d polynomial irreducible over Z_2; Sec. 3 "Ring-Specific Challenges" uses this extension
ring so that the batched check is sound; Sec. 5 fixes l = 64, d = 64.

Reading (the paper names no f): f is monic with 0/1 coefficients and irreducible mod 2, which makes
Z_2^l[x]/f the Galois ring GR(2^l, d).  For d = 64 we take f = x^64 + x^4 + x^3 + x + 1.
``is_irreducible_mod2`` re-checks irreducibility with Rabin's test at construction.

An element is a numpy uint64 array whose last axis holds the d coefficients (index c is the
coefficient of x^c), each reduced mod 2^l.  All functions broadcast over leading axes.

Pins (tests/test_oracle_galois.py): ring axioms on random elements; products against sympy's
polynomial remainder over Z; reduction mod 2 against an independent carry-less GF(2^d) product;
Frobenius a^(2^d) == a mod 2; Newton inverse a * a^-1 == 1; sympy irreducibility of f.
"""
from __future__ import annotations

import numpy as np

# f = x^64 + x^4 + x^3 + x + 1: exponents of the non-leading terms with coefficient 1.
F64_LOW_TAPS = (0, 1, 3, 4)


def _poly_mod2_mulmod(a: int, b: int, f: int) -> int:
    """Carry-less product a*b mod f over GF(2) (polynomials as Python ints, bit i = x^i)."""
    deg_f = f.bit_length() - 1
    a = _poly_mod2_rem(a, f)
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if (a >> deg_f) & 1:
            a ^= f
    return r


def _poly_mod2_rem(a: int, f: int) -> int:
    deg_f = f.bit_length() - 1
    while a and a.bit_length() - 1 >= deg_f:
        a ^= f << (a.bit_length() - 1 - deg_f)
    return a


def _poly_mod2_gcd(a: int, b: int) -> int:
    while b:
        a, b = b, _poly_mod2_rem(a, b)
    return a


def is_irreducible_mod2(f: int) -> bool:
    """Rabin's irreducibility test for f in GF(2)[x] (bit i of ``f`` = coefficient of x^i)."""
    n = f.bit_length() - 1
    if n < 1:
        return False
    x = 0b10

    def x_pow_2k(k: int) -> int:
        r = x
        for _ in range(k):
            r = _poly_mod2_mulmod(r, r, f)
        return r

    if x_pow_2k(n) != _poly_mod2_rem(x, f):
        return False
    primes = [p for p in range(2, n + 1) if n % p == 0 and all(p % q for q in range(2, p))]
    for p in primes:
        h = x_pow_2k(n // p) ^ _poly_mod2_rem(x, f)
        if _poly_mod2_gcd(f, h) != 1:
            return False
    return True


class GR:
    """Arithmetic in GR(2^l, d) with modulus f = x^d + sum_{s in low_taps} x^s."""

    def __init__(self, ell: int = 64, d: int = 64, low_taps=F64_LOW_TAPS):
        assert 1 <= ell <= 64 and d >= 1
        self.ell = ell
        self.d = d
        self.low_taps = tuple(sorted(low_taps))
        assert all(0 <= s < d for s in self.low_taps)
        self.mask = np.uint64((1 << ell) - 1) if ell < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
        f_int = (1 << d) | sum(1 << s for s in self.low_taps)
        if not is_irreducible_mod2(f_int):
            raise ValueError("f is not irreducible mod 2")
        self.f_int = f_int

    # ---- constructors -------------------------------------------------------------------------
    def zeros(self, shape=()) -> np.ndarray:
        return np.zeros(tuple(shape) + (self.d,), dtype=np.uint64)

    def const(self, c: int) -> np.ndarray:
        """The element with free coefficient c (Sec. 3: points 0, 1, 2 are these constants)."""
        e = self.zeros()
        e[0] = np.uint64(c % (1 << 64)) & self.mask
        return e

    def x(self) -> np.ndarray:
        """The class of the indeterminate x."""
        e = self.zeros()
        if self.d == 1:
            # x == -(sum of low taps) when d == 1
            e[0] = np.uint64((-len(self.low_taps)) % (1 << 64)) & self.mask
        else:
            e[1] = np.uint64(1)
        return e

    def lift(self, s: np.ndarray) -> np.ndarray:
        """Lift Z_2^l values to GR by putting them in the free coefficient, zero elsewhere.

        Fig. MTP / Sec. 3: "the free coefficient ... is set to the original shares, while the
        remaining coefficients are padded with zero shares"."""
        s = np.asarray(s, dtype=np.uint64)
        out = np.zeros(s.shape + (self.d,), dtype=np.uint64)
        out[..., 0] = s & self.mask
        return out

    # ---- ring operations ----------------------------------------------------------------------
    def add(self, a, b):
        return (np.asarray(a, dtype=np.uint64) + np.asarray(b, dtype=np.uint64)) & self.mask

    def sub(self, a, b):
        return (np.asarray(a, dtype=np.uint64) - np.asarray(b, dtype=np.uint64)) & self.mask

    def neg(self, a):
        return (np.uint64(0) - np.asarray(a, dtype=np.uint64)) & self.mask

    def scale(self, a, s):
        """Multiply by the Z_2^l scalar s (broadcast over the coefficient axis)."""
        s = np.asarray(s, dtype=np.uint64)
        return (np.asarray(a, dtype=np.uint64) * s[..., None]) & self.mask

    def reduce(self, prod: np.ndarray) -> np.ndarray:
        """Reduce a polynomial with 2d-1 coefficients modulo f (x^d = -sum_{taps} x^s)."""
        d = self.d
        prod = prod.copy()
        for k in range(prod.shape[-1] - 1, d - 1, -1):
            top = prod[..., k].copy()
            for s in self.low_taps:
                prod[..., k - d + s] -= top
            prod[..., k] = 0
        return prod[..., :d] & self.mask

    def mul(self, a, b) -> np.ndarray:
        """Schoolbook product of two elements followed by reduction mod f."""
        a = np.asarray(a, dtype=np.uint64)
        b = np.asarray(b, dtype=np.uint64)
        a, b = np.broadcast_arrays(a, b)
        d = self.d
        prod = np.zeros(a.shape[:-1] + (2 * d - 1,), dtype=np.uint64)
        for i in range(d):
            prod[..., i:i + d] += a[..., i:i + 1] * b
        return self.reduce(prod)

    def pow(self, a, e: int) -> np.ndarray:
        r = self.const(1)
        base = np.asarray(a, dtype=np.uint64)
        while e:
            if e & 1:
                r = self.mul(r, base)
            base = self.mul(base, base)
            e >>= 1
        return r

    def powers(self, a, n: int) -> np.ndarray:
        """[a^0, a^1, ..., a^(n-1)] (shape (n, d)), by doubling blocks: once a^0 .. a^(k-1) are
        known, a^(k+i) = a^i a^k for i < k."""
        out = self.zeros((n,))
        if n == 0:
            return out
        out[0] = self.const(1)
        k = 1
        ak = np.asarray(a, dtype=np.uint64) & self.mask        # a^k
        while k < n:
            m = min(k, n - k)
            out[k:k + m] = self.mul(out[:m], ak)
            ak = self.mul(ak, ak)
            k += m
        return out

    def is_unit(self, a) -> bool:
        """a is a unit iff its reduction mod 2 is non-zero in GF(2^d) = GR / 2GR."""
        return bool(np.any(np.asarray(a) & np.uint64(1)))

    def inv(self, a) -> np.ndarray:
        """Inverse of a unit: GF(2^d) inverse by exponentiation, then Newton (Hensel) lifting
        y <- y (2 - a y), which doubles the number of correct 2-adic digits per step."""
        a = np.asarray(a, dtype=np.uint64)
        if not self.is_unit(a):
            raise ZeroDivisionError("not a unit of GR(2^l, d)")
        a_bits = sum(int(a[c] & np.uint64(1)) << c for c in range(self.d))
        # a^(2^d - 2) in GF(2^d)
        y_bits, base, e = 1, a_bits, (1 << self.d) - 2
        while e:
            if e & 1:
                y_bits = _poly_mod2_mulmod(y_bits, base, self.f_int)
            base = _poly_mod2_mulmod(base, base, self.f_int)
            e >>= 1
        y = self.zeros()
        for c in range(self.d):
            y[c] = np.uint64((y_bits >> c) & 1)
        two = self.const(2)
        for _ in range(7):  # 1 -> 2 -> ... -> 128 >= 64 correct bits
            y = self.mul(y, self.sub(two, self.mul(a, y)))
        assert np.array_equal(self.mul(a, y), self.const(1))
        return y

    def sum(self, a, axis=0) -> np.ndarray:
        return np.sum(np.asarray(a, dtype=np.uint64), axis=axis, dtype=np.uint64) & self.mask

    def inner(self, a, b) -> np.ndarray:
        """sum_i a_i * b_i over the leading axis."""
        if len(a) == 0:
            return self.zeros()
        return self.sum(self.mul(a, b), axis=0)


GR64 = None


def gr64() -> GR:
    """The ring used throughout the paper's benchmarks: l = 64, d = 64 (Sec. 5)."""
    global GR64
    if GR64 is None:
        GR64 = GR(64, 64, F64_LOW_TAPS)
    return GR64
