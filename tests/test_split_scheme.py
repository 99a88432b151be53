"""The arithmetic behind the long-contraction split-TF32 products, checked on
the CPU with a numpy model (no GPU, no kernel code).

Each element of a row of op(A) (a column of op(B)) within a 64-wide K group
is rounded to the grid 2^(T-31) of the group's largest exponent T and cut
into integer slices of 9, 11 and 11 bits.  The claims the kernel rests on:
1. every slice is exactly an FP32 (indeed TF32) value;
2. the 64 hi*hi products of a group sum exactly in FP32 whatever the order
   (all are multiples of one unit and the total stays below 2^24 units);
3. summing the eight retained products (all but lo*lo) leaves an error of
   about 2^-32 max|a| max|b| per term.
"""
import numpy as np

G = 64


def slices(v, T):
    """hi, mid, lo of v on the grid 2^(T-31) (v within 2^T in magnitude)."""
    q = np.rint(np.abs(v) * 2.0 ** (31 - T)).astype(np.int64)
    s = np.sign(v)
    hi, mid, lo = q >> 22, (q >> 11) & 0x7FF, q & 0x7FF
    return (s * hi * 2.0 ** (T - 9), s * mid * 2.0 ** (T - 20), s * lo * 2.0 ** (T - 31)), (hi, mid, lo)


def group_exponent(x):
    """T with max|x| < 2^T (the kernel's biased exponent eg minus 1022)."""
    m = np.max(np.abs(x))
    return int(np.frexp(m)[1]) if m > 0 else 0


def test_slices_are_exact_tf32_and_reassemble():
    rng = np.random.default_rng(1)
    # within the FP32 exponent range (the split products' documented input range)
    for scale in (1.0, 1e-25, 1e30, 3.7):
        x = rng.standard_normal(G) * scale
        T = group_exponent(x)
        (h, m, l), (qh, qm, ql) = slices(x, T)
        assert np.all(qh <= 2 ** 9) and np.all(qm < 2 ** 11) and np.all(ql < 2 ** 11)
        for part in (h, m, l):
            # representable in FP32 with at most 11 significant bits (TF32)
            np.testing.assert_array_equal(part.astype(np.float32).astype(np.float64), part)
        assert np.max(np.abs(h + m + l - x)) <= 2.0 ** (T - 32) * (1 + 1e-12)


def test_hi_products_sum_exactly_in_fp32_in_any_order():
    rng = np.random.default_rng(2)
    for _ in range(20):
        a, b = rng.standard_normal(G), rng.standard_normal(G)
        (ha, _, _), _ = slices(a, group_exponent(a))
        (hb, _, _), _ = slices(b, group_exponent(b))
        prods = (ha * hb).astype(np.float32)          # each product exact in FP32 (<= 18 bits)
        np.testing.assert_array_equal(prods.astype(np.float64), ha * hb)
        exact = np.sum(ha * hb)                        # FP64, exact here
        for _ in range(5):
            acc = np.float32(0.0)
            for p in rng.permutation(prods):
                acc = np.float32(acc + p)
            assert float(acc) == exact


def test_eight_products_error_bound():
    rng = np.random.default_rng(3)
    K = 4 * G
    for _ in range(10):
        a, b = rng.standard_normal(K), rng.standard_normal(K)
        total = 0.0
        bound = 0.0
        for g0 in range(0, K, G):
            ag, bg = a[g0:g0 + G], b[g0:g0 + G]
            Ta, Tb = group_exponent(ag), group_exponent(bg)
            (ah, am, al), _ = slices(ag, Ta)
            (bh, bm, bl), _ = slices(bg, Tb)
            hh = np.float32(np.sum(ah * bh))           # exact, as above
            rest = np.float32(0.0)
            for p in (ah * bm, am * bh, ah * bl, am * bm, al * bh, am * bl, al * bm):
                for v in p.astype(np.float32):
                    rest = np.float32(rest + v)
            total += float(hh) + float(rest)           # drained into a compensated sum
            bound += G * 2.0 ** (Ta + Tb - 32)
        err = abs(total - float(a @ b))
        assert err <= 4 * bound, (err, bound)
        assert err <= 1e-8 * np.sum(np.abs(a) * np.abs(b)) * 8
