"""Host-side test of the integer-pipe binary64 multiplication used by the
stage kernels (csrc/fp64_int.cuh): general products, products with powers of
two and with small odd integers times powers of two.  The header also compiles as plain C++;
here it is built with g++ and every product is compared, bit for bit, with the
IEEE 754 round-to-nearest-even product of the host (numpy), including signed
zeros, ties, and the cases handed back to the FP64 unit (subnormal, infinite
and NaN operands, overflow and results below the normal range)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

LIB = None
CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1604_03360_gb300", "csrc")

SRC = r'''
#include "fp64_int.cuh"
using namespace hydro;
extern "C" void mul_batch(const double* a, const double* b, double* out, long n, int* fast)
{
    for (long i = 0; i < n; ++i) {
        uint64_t r;
        fast[i] = dmul_int_bits(f64_to_bits(a[i]), f64_to_bits(b[i]), r) ? 1 : 0;
        out[i] = dmul_int(a[i], b[i]);
    }
}
template <int CB>
static void small_cb(const double* a, double* out, long n, int* fast, unsigned c, int k, double f)
{
    for (long i = 0; i < n; ++i) {
        uint64_t r;
        const bool ok = dmul_small_bits<CB>(f64_to_bits(a[i]), c, k, r);
        fast[i] = ok ? 1 : 0;
        out[i] = ok ? f64_from_bits(r) : a[i] * f;
    }
}
extern "C" void small_batch(const double* a, double* out, long n, int* fast, unsigned c, int cb, int k, double f)
{
    switch (cb) {
    case 2: small_cb<2>(a, out, n, fast, c, k, f); break;
    case 3: small_cb<3>(a, out, n, fast, c, k, f); break;
    case 6: small_cb<6>(a, out, n, fast, c, k, f); break;
    case 7: small_cb<7>(a, out, n, fast, c, k, f); break;
    case 10: small_cb<10>(a, out, n, fast, c, k, f); break;
    }
}
extern "C" void pow2_batch(const double* a, double* out, long n, int* fast, int k, double f)
{
    for (long i = 0; i < n; ++i) {
        uint64_t r;
        const bool ok = dmul_pow2_bits(f64_to_bits(a[i]), k, r);
        fast[i] = ok ? 1 : 0;
        out[i] = ok ? f64_from_bits(r) : a[i] * f;
    }
}
extern "C" void templ_batch(const double* a, double* out, long n)
{
    // the typed wrappers used by the kernels
    for (long i = 0; i < n; ++i) {
        out[6 * i + 0] = xmul_pow2<true, -2>(a[i]);
        out[6 * i + 1] = xmul_pow2<true, 1>(a[i]);
        out[6 * i + 2] = xmul_small<true, 3, 2, -1>(a[i]);
        out[6 * i + 3] = xmul_small<true, 39, 6, 0>(a[i]);
        out[6 * i + 4] = xmul<true>(781.0 / 20.0, a[i]);
        out[6 * i + 5] = xmul<true>(-1.0 / 3.0, a[i]);
    }
}
'''


@pytest.fixture(scope="module")
def mul(tmp_path_factory):
    d = tmp_path_factory.mktemp("fp64int")
    src = d / "t.cpp"
    src.write_text(SRC)
    so = d / "t.so"
    # -ffp-contract=off: the fallback product must be a plain IEEE multiplication
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC, str(src), "-o",
                    str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    lib.mul_batch.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_long, ctypes.c_void_p]
    global LIB
    LIB = lib

    def run(a, b):
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        out = np.empty_like(a)
        fast = np.empty(a.shape, dtype=np.int32)
        lib.mul_batch(a.ctypes.data, b.ctypes.data, out.ctypes.data, a.size, fast.ctypes.data)
        return out, fast
    return run


def from_fields(sign, exp, man):
    bits = (sign.astype(np.uint64) << np.uint64(63)) | (exp.astype(np.uint64) << np.uint64(52)) | \
        (man.astype(np.uint64) & np.uint64((1 << 52) - 1))
    return bits.view(np.float64)


def check(mul, a, b):
    got, fast = mul(a, b)
    with np.errstate(all="ignore"):
        ref = a * b
    gb, rb = got.view(np.uint64), ref.view(np.uint64)
    same = (gb == rb) | (np.isnan(got) & np.isnan(ref))
    bad = np.flatnonzero(~same)
    assert bad.size == 0, [(a[i], b[i], got[i], ref[i]) for i in bad[:5]]
    return fast


def test_random_bit_patterns(mul):
    rng = np.random.default_rng(1)
    a = rng.integers(0, 2 ** 64, 1_000_000, dtype=np.uint64, endpoint=False).view(np.float64)
    b = rng.integers(0, 2 ** 64, 1_000_000, dtype=np.uint64, endpoint=False).view(np.float64)
    check(mul, a, b)


def test_random_normals_take_the_integer_path(mul):
    rng = np.random.default_rng(2)
    n = 2_000_000
    a = from_fields(rng.integers(0, 2, n), rng.integers(600, 1400, n), rng.integers(0, 2 ** 52, n, dtype=np.uint64))
    b = from_fields(rng.integers(0, 2, n), rng.integers(600, 1400, n), rng.integers(0, 2 ** 52, n, dtype=np.uint64))
    fast = check(mul, a, b)
    assert fast.all()


def test_exponent_range_boundaries(mul):
    """Products at the edges of the normal range: the integer path must either
    be exact or hand over (overflow, subnormal results)."""
    rng = np.random.default_rng(3)
    n = 400_000
    man_a = rng.integers(0, 2 ** 52, n, dtype=np.uint64)
    man_b = rng.integers(0, 2 ** 52, n, dtype=np.uint64)
    for target in (-3, -1, 0, 1, 2, 2045, 2046, 2047, 2048):
        ea = rng.integers(1, 2047, n)
        eb = np.clip(target + 1023 - ea, 1, 2046)
        fast = check(mul, from_fields(rng.integers(0, 2, n), ea, man_a), from_fields(rng.integers(0, 2, n), eb, man_b))
        if 3 <= target <= 2044:
            assert fast.all()
    # the smallest normal reached by rounding up from just below it
    a = np.array([np.nextafter(1.0, 0.0), 2.0 ** -1022 * (2 - 2.0 ** -52)])
    b = np.array([2.0 ** -1022, np.nextafter(0.5, 1.0)])
    check(mul, a, b)


def test_short_significands_exercise_ties_and_exact_products(mul):
    """Significands with few bits give exact products, carries out of the
    rounding and exact ties (round half to even)."""
    rng = np.random.default_rng(4)
    n = 1_000_000
    out_fast = []
    for k in (1, 2, 3, 8, 20, 27, 30, 40):
        ma = (rng.integers(0, 2 ** k, n, dtype=np.uint64) << np.uint64(52 - k)) if k <= 52 else None
        mb = (rng.integers(0, 2 ** k, n, dtype=np.uint64) << np.uint64(52 - k))
        # odd significand patterns around the tie position
        mb2 = mb | np.uint64(1)
        e = rng.integers(900, 1100, n)
        out_fast.append(check(mul, from_fields(rng.integers(0, 2, n), e, ma), from_fields(rng.integers(0, 2, n), e, mb2)))
        out_fast.append(check(mul, from_fields(rng.integers(0, 2, n), e, ma), from_fields(rng.integers(0, 2, n), e, mb)))
    # (1 + 2^-52)(1 + 2^-1 + 2^-52 j): the product sits exactly half-way for suitable j
    j = np.arange(0, 4096, dtype=np.uint64)
    a = from_fields(np.zeros(j.size, int), np.full(j.size, 1023), np.full(j.size, 1, np.uint64))
    b = from_fields(np.zeros(j.size, int), np.full(j.size, 1023), (np.uint64(1) << np.uint64(51)) | j)
    out_fast.append(check(mul, a, b))
    assert np.concatenate(out_fast).all()


def test_zeros_and_specials(mul):
    vals = np.array([0.0, -0.0, 1.0, -1.5, np.inf, -np.inf, np.nan, 5e-324, -2.0 ** -1060, 2.0 ** -1022, 1.7e308,
                     3.0, -7.25e-200])
    a, b = np.meshgrid(vals, vals)
    fast = check(mul, a.ravel(), b.ravel())
    # finite x zero is decided on the integer path
    fin = np.isfinite(a.ravel()) & np.isfinite(b.ravel()) & ((a.ravel() == 0) | (b.ravel() == 0))
    assert fast[fin].all()


def test_exact_ties_round_to_even(mul):
    """Odd significands of 27 and 28 bits multiply to an odd 54- or 55-bit
    integer; when it has 54 bits the 53-bit result lies exactly half-way
    between two neighbours and must round to the even one."""
    rng = np.random.default_rng(5)
    n = 200_000
    m1 = rng.integers(2 ** 25, 2 ** 26, n, dtype=np.uint64) * np.uint64(2) + np.uint64(1)   # odd, 27 bits
    m2 = rng.integers(2 ** 26, 2 ** 27, n, dtype=np.uint64) * np.uint64(2) + np.uint64(1)   # odd, 28 bits
    e = rng.integers(900, 1100, n)
    a = from_fields(rng.integers(0, 2, n), e, m1 << np.uint64(26))
    b = from_fields(rng.integers(0, 2, n), e, m2 << np.uint64(25))
    ties = sum(1 for x, y in zip(m1[:20000].tolist(), m2[:20000].tolist()) if (x * y).bit_length() == 54)
    assert ties > 5000
    assert check(mul, a, b).all()


def _lib(mul):
    return LIB


def test_small_odd_factors_and_powers_of_two(mul):
    lib = _lib(mul)
    rng = np.random.default_rng(6)
    n = 1_000_000
    a = from_fields(rng.integers(0, 2, n), rng.integers(1, 2047, n), rng.integers(0, 2 ** 52, n, dtype=np.uint64))
    a[:1000] = rng.standard_normal(1000)
    a[1000:1010] = [0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -1e-310, 2.0 ** -1022, 1.7e308, -2.0 ** 1023]
    out = np.empty_like(a)
    fast = np.empty(n, dtype=np.int32)
    lib.small_batch.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p, ctypes.c_uint,
                                ctypes.c_int, ctypes.c_int, ctypes.c_double]
    lib.pow2_batch.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p, ctypes.c_int,
                               ctypes.c_double]
    for c, cb in ((3, 2), (5, 3), (7, 3), (39, 6), (101, 7), (1021, 10)):
        for k in (-3, -1, 0, 2):
            f = c * 2.0 ** k
            lib.small_batch(a.ctypes.data, out.ctypes.data, n, fast.ctypes.data, c, cb, k, f)
            with np.errstate(all="ignore"):
                ref = a * f
            same = (out.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(out) & np.isnan(ref))
            assert same.all(), (c, k, a[~same][:3])
            assert fast[1010:].mean() > 0.99
    for k in (-2, -1, 1, 3):
        f = 2.0 ** k
        lib.pow2_batch(a.ctypes.data, out.ctypes.data, n, fast.ctypes.data, k, f)
        with np.errstate(all="ignore"):
            ref = a * f
        same = (out.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(out) & np.isnan(ref))
        assert same.all(), (k, a[~same][:3])


def test_typed_wrappers(mul):
    lib = _lib(mul)
    rng = np.random.default_rng(8)
    a = np.concatenate([rng.standard_normal(100000) * 10.0 ** rng.uniform(-30, 30, 100000), [0.0, -0.0]])
    out = np.empty(6 * a.size)
    lib.templ_batch.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long]
    lib.templ_batch(a.ctypes.data, out.ctypes.data, a.size)
    out = out.reshape(-1, 6)
    ref = np.stack([a * 0.25, a * 2.0, a * 1.5, a * 39.0, (781.0 / 20.0) * a, (-1.0 / 3.0) * a], axis=1)
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))
