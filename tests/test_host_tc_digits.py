"""Arithmetic of the tensor-core Schur products (FP32 pairs), checked on the
host: the fixed-point digit split (Ozaki, Ogita, Oishi and Rump, Numer.
Algorithms 59 (2012)) that the GEMM kernel relies on, restated here in numpy
float32 with the kernel's operation order:

* every real x of a row with scale 2^e (|Re| + |Im| < 2^e) becomes
  X = round(x 2^(54 - e)) as 7 balanced base-256 digits, d_t in [-128, 127]
  for t >= 1 and |d_0| <= 64, formed separately for the hi and lo parts of an
  FP32 pair and carried;
* the digits of Re + Im are the carried sums of the digits of Re and Im, so
  they represent X_re + X_im exactly;
* the FP32 sums of the digit-sum groups g = 0 .. 3 over a chunk of 320 k
  stay below 2^24, the bound under which the tensor cores add them exactly;
  the groups 4, 5, 6 share one FP32 accumulator (each product weighted
  2^(-8g)), whose rounding is emulated here in float32;
* the dropped pairs (t + t' >= 7), the rounding to 54 bits and the shared
  accumulator leave a normwise error of order 2^-52 max|a| max|b| k per entry.

No GPU and no library call: the kernel's own results are covered by the GPU
parity tests.
"""
import numpy as np

F = np.float32
S, FBITS, CHUNK_K, NACC = 7, 54, 320, 5


def rint(x):
    return F(np.rint(F(x)))


def digits(V):
    """Balanced base-256 digits of an integer-valued float32 V, d[6] least significant."""
    V = rint(V)
    d = [F(0)] * S
    for t in range(S - 1, 0, -1):
        q = rint(F(V * F(0.00390625)))
        r = F(float(V) - 256.0 * float(q))  # exact: |r| <= 128
        up = F(1) if r >= 128 else F(0)
        d[t] = F(r - F(256) * up)
        V = F(q + up)
    d[0] = V
    return d


def carry(d):
    d = list(d)
    for t in range(S - 1, 0, -1):
        c = rint(F(d[t] * F(0.00390625)))
        r = F(d[t] - F(256) * c)
        up = F(1) if r >= 128 else F(0)
        d[t] = F(r - F(256) * up)
        d[t - 1] = F(d[t - 1] + c + up)
    return d


def value(d):
    return sum(int(v) * 256 ** (S - 1 - t) for t, v in enumerate(d))


def split_pair(hi, lo, sc):
    """Digits of the FP32 pair hi + lo scaled by sc (a power of two)."""
    return carry([a + b for a, b in zip(digits(F(hi * sc)), digits(F(lo * sc)))])


def _pairs(rng, n):
    e = rng.integers(-30, 30, size=n)
    x = rng.uniform(-1, 1, size=n) * np.exp2(e) / 1.0001
    y = rng.uniform(-1, 1, size=n) * np.exp2(e) / 1.0001 * (1 - np.abs(x) / np.exp2(e))
    return e, x, y


def test_digit_ranges_and_exact_reconstruction():
    rng = np.random.default_rng(1305)
    e, x, y = _pairs(rng, 4000)
    for i in range(len(e)):
        sc = F(2.0 ** (FBITS - int(e[i])))
        hx = F(x[i]); lx = F(x[i] - float(hx))
        hy = F(y[i]); ly = F(y[i] - float(hy))
        r = split_pair(hx, lx, sc)
        im = split_pair(hy, ly, sc)
        s = carry([a + b for a, b in zip(r, im)])
        # X = round(hi sc) + round(lo sc): the pair to 54 bits below the row scale
        assert value(r) == int(np.rint(float(hx) * float(sc))) + int(np.rint(float(F(lx * sc))))
        assert value(s) == value(r) + value(im)
        for d in (r, im, s):
            assert all(-128 <= v <= 127 for v in d[1:])
            assert abs(d[0]) <= 64
            # every digit is exact in BF16 (8 significant bits)
            assert all(float(v) == float(np.float32(v)) and abs(v) <= 256 for v in d)


def test_group_sums_stay_exact_over_a_chunk():
    """Worst case of the exact groups g = 0 .. 3 over CHUNK_K terms: pairs of two
    digits of magnitude 128, those with the top digit 64 x 128."""
    worst = {0: 64 * 64, 1: 2 * 64 * 128, 2: 2 * 64 * 128 + 128 * 128, 3: 2 * 64 * 128 + 2 * 128 * 128}
    for g, per_k in worst.items():
        assert CHUNK_K * per_k < 2 ** 24, (g, CHUNK_K * per_k)
    # the bound the kernel asserts: 3 * 2^14 per k for every exact group
    assert max(worst.values()) <= 3 * 2 ** 14 and CHUNK_K * 3 * 2 ** 14 < 2 ** 24


def test_truncated_digit_product_error_bound():
    """Complex dot products through the digits (3 real products, pairs t + t' < 7;
    groups 0 .. 3 summed exactly, groups 4..6 in one float32 accumulator with the
    weights 2^(-8g), in the MMAs' order: 16 k per product, pair by pair) against
    float64.  Per term and real product: rounding each factor to 54 bits below
    its scale costs at most 2 * 2^(ea + eb - 54); the dropped pairs at most
    sum_{g >= 7} (13 - g) 2^14 256^(12 - g) 2^(ea + eb - 108) < 2^(ea + eb - 51.3);
    the shared accumulator's rounding at most 2^-24 of its magnitude per
    addition (< 2^(ea + eb - 48) per term); three real products: below
    k 2^(ea + eb - 45) in all."""
    rng = np.random.default_rng(7)
    k = 48
    a = (rng.standard_normal(k) + 1j * rng.standard_normal(k)) * np.exp2(rng.integers(-6, 1, size=k))
    b = (rng.standard_normal(k) + 1j * rng.standard_normal(k)) * np.exp2(rng.integers(-6, 1, size=k))
    ea = int(np.floor(np.log2(np.max(np.abs(a.real) + np.abs(a.imag)) * 1.0001))) + 1
    eb = int(np.floor(np.log2(np.max(np.abs(b.real) + np.abs(b.imag)) * 1.0001))) + 1

    def dig(v, e):
        sc = F(2.0 ** (FBITS - e))
        h = F(v); lo = F(v - float(h))
        return split_pair(h, lo, sc)

    comp = []
    for vec, e in ((a, ea), (b, eb)):
        re = [dig(v.real, e) for v in vec]
        im = [dig(v.imag, e) for v in vec]
        sm = [carry([p + q for p, q in zip(x, y)]) for x, y in zip(re, im)]
        comp.append((re, im, sm))
    P = []
    for c in range(3):
        exact = 0          # groups 0..3, exact integers in units of 2^-24 (2^(-8g) weights)
        shared = F(0)      # groups 4..6 in float32, weights 2^(-8g)
        for k0 in range(0, k, 16):
            for t1 in range(S):
                for t2 in range(S - t1):
                    g = t1 + t2
                    Dg = sum(int(comp[0][c][q][t1]) * int(comp[1][c][q][t2]) for q in range(k0, min(k, k0 + 16)))
                    if g < NACC - 1:
                        exact += Dg * 256 ** (NACC - 2 - g)
                    else:
                        shared = F(shared + F(Dg * 2.0 ** (-8 * g)))
        # sum_g 2^(-8g) D_g; times 256^12 for the integer scale of the digits
        P.append(exact * 2.0 ** (-8 * (NACC - 2)) + float(shared))
    scale = 2.0 ** (ea + eb - 2 * FBITS) * 256.0 ** 12
    got = complex((P[0] - P[1]) * scale, (P[2] - P[0] - P[1]) * scale)
    ref = np.dot(a, b)
    bound = k * 2.0 ** (ea + eb - 45)
    err = abs(got - ref)
    assert err <= bound, (err, bound)
    # far below single precision: the scheme carries FP32-pair accuracy
    assert err <= 1e-13 * np.sum(np.abs(a) * np.abs(b))
