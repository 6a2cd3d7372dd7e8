"""Arithmetic of the tensor-core Schur products (FP32 pairs), checked on the
host: the fixed-point digit split (Ozaki, Ogita, Oishi and Rump, Numer.
Algorithms 59 (2012)) that the GEMM kernel relies on, restated here in numpy
float32 and Python integers with the kernel's operation order:

* every real x = h + l (an FP32 pair) of a row with scale 2^e
  (|Re| + |Im| < 2^e) becomes the integer X = round(h 2^(54 - e)) +
  round(l 2^(54 - e)), written as 7 balanced base-256 digits, d_t in
  [-128, 127] for t >= 1 and |d_0| <= 64: the bytes of X + sum_b 128 256^b,
  less 128 each;
* the digits of Re + Im are those of the integer X_re + X_im;
* the kernel stores each digit as a two's-complement byte and moves bytes
  between elements and digit planes with byte permutations, emulated here;
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
BIAS = sum(128 * 256 ** b for b in range(S))


def fixed(hi, lo, sc):
    """X = round(hi sc) + round(lo sc), each rounded to nearest even (sc a power of two)."""
    return int(np.rint(float(F(hi * sc)))) + int(np.rint(float(F(lo * sc))))


def digits(X):
    """Balanced base-256 digits of |X| < 2^54, d[0] most significant."""
    Y = X + BIAS
    assert 0 <= Y < 2 ** 56
    return [((Y >> (8 * (S - 1 - t))) & 0xFF) - 128 for t in range(S)]


def value(d):
    return sum(int(v) * 256 ** (S - 1 - t) for t, v in enumerate(d))


def byte_perm(x, y, sel):
    """CUDA __byte_perm without the sign-replication mode: byte i of the result
    is byte (nibble i of sel) of the 8 bytes x (0..3), y (4..7)."""
    src = (int(x) & 0xFFFFFFFF) | ((int(y) & 0xFFFFFFFF) << 32)
    return sum(((src >> (8 * ((sel >> (4 * i)) & 7))) & 0xFF) << (8 * i) for i in range(4))


def transpose4(w):
    t0, t1 = byte_perm(w[0], w[1], 0x5140), byte_perm(w[0], w[1], 0x7362)
    t2, t3 = byte_perm(w[2], w[3], 0x5140), byte_perm(w[2], w[3], 0x7362)
    return [byte_perm(t0, t2, 0x5410), byte_perm(t0, t2, 0x7632), byte_perm(t1, t3, 0x5410),
            byte_perm(t1, t3, 0x7632)]


def byte_image(xs):
    """The kernel's digit planes of 8 integers: plane t, word g, byte q holds digit
    t of element 4g + q as a two's-complement byte."""
    mask = (1 << 64) - 1
    y = [((X + 0x80808080808080) & mask) ^ 0x80808080808080 for X in xs]
    lo = [v & 0xFFFFFFFF for v in y]
    hi = [(v >> 32) & 0xFFFFFFFF for v in y]
    w = [[0, 0] for _ in range(S)]
    for g in range(2):
        ol = transpose4(lo[4 * g:4 * g + 4])
        oh = transpose4(hi[4 * g:4 * g + 4])
        for b in range(4):
            w[S - 1 - b][g] = ol[b]
        for b in range(3):
            w[S - 5 - b][g] = oh[b]
    return w


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
        xr, xi = fixed(hx, lx, sc), fixed(hy, ly, sc)
        assert abs(xr) < 2 ** 54 and abs(xi) < 2 ** 54 and abs(xr + xi) < 2 ** 54
        r, im, s = digits(xr), digits(xi), digits(xr + xi)
        # X = round(hi sc) + round(lo sc): the pair to 54 bits below the row scale
        assert value(r) == xr and value(im) == xi and value(s) == xr + xi
        assert abs(xr - (float(hx) + float(lx)) * 2.0 ** (FBITS - int(e[i]))) <= 1.0
        for d in (r, im, s):
            assert all(-128 <= v <= 127 for v in d[1:])
            assert abs(d[0]) <= 64
            # every digit is exact in BF16 (8 significant bits)
            assert all(float(v) == float(np.float32(v)) and abs(v) <= 256 for v in d)


def test_byte_image_of_the_digit_planes():
    """The kernel's byte permutations put digit t of element q at byte q of plane
    t, in two's complement, for integers across the whole range (extremes
    included)."""
    rng = np.random.default_rng(11)
    lim = 2 ** 54 - 1
    cases = [[lim, -lim, 0, 1, -1, 2 ** 47, -(2 ** 47) - 5, 127]]
    cases += [[int(v) for v in rng.integers(-lim, lim, size=8, dtype=np.int64)] for _ in range(200)]
    cases += [[int(v) for v in rng.integers(-2 ** 20, 2 ** 20, size=8)] for _ in range(50)]
    for xs in cases:
        w = byte_image(xs)
        for q, X in enumerate(xs):
            d = digits(X)
            for t in range(S):
                b = (w[t][q // 4] >> (8 * (q % 4))) & 0xFF
                assert (b - 256 if b >= 128 else b) == d[t], (X, q, t)


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

    def fix(v, e):
        sc = F(2.0 ** (FBITS - e))
        h = F(v); lo = F(v - float(h))
        return fixed(h, lo, sc)

    comp = []
    for vec, e in ((a, ea), (b, eb)):
        xr = [fix(v.real, e) for v in vec]
        xi = [fix(v.imag, e) for v in vec]
        comp.append(([digits(v) for v in xr], [digits(v) for v in xi], [digits(p + q) for p, q in zip(xr, xi)]))
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
