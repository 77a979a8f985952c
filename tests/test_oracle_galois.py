"""Pins for oracle.galois against sympy and independent carry-less arithmetic (no GPU)."""
import numpy as np
import pytest
import sympy

from oracle.galois import GR, F64_LOW_TAPS, gr64, is_irreducible_mod2

U64 = np.uint64
MASK = (1 << 64) - 1


def test_f64_irreducible_sympy_and_rabin():
    x = sympy.symbols("x")
    f = x**64 + x**4 + x**3 + x + 1
    assert sympy.Poly(f, x, modulus=2).is_irreducible
    assert is_irreducible_mod2((1 << 64) | 0b11011)


def test_rabin_agrees_with_sympy_small_degrees():
    x = sympy.symbols("x")
    rng = np.random.default_rng(0)
    for _ in range(60):
        deg = int(rng.integers(2, 12))
        f = (1 << deg) | int(rng.integers(0, 1 << deg))
        expr = sum(x**i for i in range(deg + 1) if (f >> i) & 1)
        assert is_irreducible_mod2(f) == sympy.Poly(expr, x, modulus=2).is_irreducible


def _sympy_mul(a, b):
    """Reference product: polynomial product over Z, remainder by f over Z, coefficients mod 2^64."""
    x = sympy.symbols("x")
    f = sympy.Poly(x**64 + x**4 + x**3 + x + 1, x, domain="ZZ")
    pa = sympy.Poly(list(reversed([int(v) for v in a])), x, domain="ZZ")
    pb = sympy.Poly(list(reversed([int(v) for v in b])), x, domain="ZZ")
    rem = (pa * pb).rem(f)
    coeffs = list(reversed(rem.all_coeffs()))
    coeffs += [0] * (64 - len(coeffs))
    return np.array([int(c) % (1 << 64) for c in coeffs], dtype=U64)


def test_mul_matches_sympy_remainder():
    gr = gr64()
    rng = np.random.default_rng(1)
    for _ in range(3):
        a = rng.integers(0, 2**63, 64, dtype=U64) * U64(2) + rng.integers(0, 2, 64, dtype=U64)
        b = rng.integers(0, 2**63, 64, dtype=U64) * U64(3)
        assert np.array_equal(gr.mul(a, b), _sympy_mul(a, b))


def test_ring_axioms():
    gr = gr64()
    rng = np.random.default_rng(2)
    a, b, c = (rng.integers(0, 2**64, (8, 64), dtype=U64) for _ in range(3))
    assert np.array_equal(gr.mul(a, b), gr.mul(b, a))
    assert np.array_equal(gr.mul(gr.mul(a, b), c), gr.mul(a, gr.mul(b, c)))
    assert np.array_equal(gr.mul(a, gr.add(b, c)), gr.add(gr.mul(a, b), gr.mul(a, c)))
    assert np.array_equal(gr.mul(a, gr.const(1)), a)
    assert np.array_equal(gr.add(a, gr.neg(a)), np.zeros_like(a))


def _clmul_mod(a_bits, b_bits, f):
    r = 0
    for i in range(64):
        if (b_bits >> i) & 1:
            r ^= a_bits << i
    for k in range(126, 63, -1):
        if (r >> k) & 1:
            r ^= f << (k - 64)
    return r


def test_reduction_mod2_is_gf2_64_product():
    gr = gr64()
    f = (1 << 64) | 0b11011
    rng = np.random.default_rng(3)
    for _ in range(5):
        a = rng.integers(0, 2**64, 64, dtype=U64)
        b = rng.integers(0, 2**64, 64, dtype=U64)
        p = gr.mul(a, b)
        bits = lambda v: sum(int(v[c] & U64(1)) << c for c in range(64))
        assert bits(p) == _clmul_mod(bits(a), bits(b), f)


def test_frobenius_mod2():
    gr = gr64()
    a = np.random.default_rng(4).integers(0, 2**64, 64, dtype=U64)
    p = a.copy()
    for _ in range(64):
        p = gr.mul(p, p)
    assert np.array_equal(p & U64(1), a & U64(1))


def test_inverse_and_units():
    gr = gr64()
    rng = np.random.default_rng(5)
    a = rng.integers(0, 2**64, 64, dtype=U64)
    a[0] |= U64(1)
    assert np.array_equal(gr.mul(a, gr.inv(a)), gr.const(1))
    x = gr.x()
    one = gr.const(1)
    for u in (x, gr.sub(one, x), gr.mul(x, gr.sub(x, one))):
        assert gr.is_unit(u)
        assert np.array_equal(gr.mul(u, gr.inv(u)), one)
    assert not gr.is_unit(gr.const(2))
    with pytest.raises(ZeroDivisionError):
        gr.inv(gr.const(2))


@pytest.mark.parametrize("ell,d,taps", [(2, 2, (0, 1)), (3, 2, (0, 1)), (2, 3, (0, 1)), (4, 1, (0,))])
def test_tiny_ring_mul_bruteforce(ell, d, taps):
    """Every product in a tiny GR against integer polynomial arithmetic written here."""
    gr = GR(ell, d, taps)
    q = 1 << ell
    elems = [np.array([(v >> (ell * c)) % q for c in range(d)], dtype=U64) for v in range(q ** d)]
    for a in elems[:: max(1, len(elems) // 16)]:
        for b in elems[:: max(1, len(elems) // 16)]:
            prod = [0] * (2 * d - 1)
            for i in range(d):
                for j in range(d):
                    prod[i + j] += int(a[i]) * int(b[j])
            for k in range(2 * d - 2, d - 1, -1):
                top = prod[k]
                prod[k] = 0
                for s in taps:
                    prod[k - d + s] -= top
            ref = np.array([v % q for v in prod[:d]], dtype=U64)
            assert np.array_equal(gr.mul(a, b), ref)
