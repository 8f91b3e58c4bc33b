"""The pair arithmetic of CSS_FP64_SPLIT, restated in numpy float32 on the CPU (no GPU): every
value x as x_hi + x_lo (x_hi = fl32(x), x_lo = fl32(x - x_hi)), a product by Dekker's exact FMA
error plus the two cross terms, sums by Knuth's TwoSum into a hi + lo pair.  A block product of
the workload's shape (23 x 23 blocks times 23 rows of V, 30 neighbours, 690 terms per output) then
agrees with FP64 to about 2^-44 of the magnitude of its terms (median; at worst about 2^-40: the
FP32 roundings of the low word), against 2^-19 for a plain FP32 product."""
import numpy as np

f32 = np.float32


def split(x):
    hi = x.astype(f32)
    lo = (x - hi.astype(np.float64)).astype(f32)
    return hi, lo


def fma32(a, b, c):
    # exact in float64 for float32 operands (24 + 24 significand bits), then one rounding
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def pair_matmul(H, V):
    """W = H V term by term in the pair arithmetic (k ascending), as the kernel sums it."""
    hh, hl = split(H)
    vh, vl = split(V)
    sh = np.zeros((H.shape[0], V.shape[1]), f32)
    sl = np.zeros_like(sh)
    for k in range(H.shape[1]):
        a_h, a_l = hh[:, k:k + 1], hl[:, k:k + 1]
        b_h, b_l = vh[k:k + 1, :], vl[k:k + 1, :]
        p = (a_h * b_h).astype(f32)
        c = fma32(a_h, b_h, -p)           # exact error of the rounded product
        c = fma32(a_l, b_h, c)
        c = fma32(a_h, b_l, c)
        s = (sh + p).astype(f32)          # TwoSum(sh, p)
        bv = (s - sh).astype(f32)
        err = ((sh - (s - bv)).astype(f32) + (p - bv).astype(f32)).astype(f32)
        sl = (sl + (err + c).astype(f32)).astype(f32)
        sh = s
    return sh.astype(np.float64) + sl.astype(np.float64)


def test_dekker_product_error_is_exact():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(10000).astype(f32)
    b = rng.standard_normal(10000).astype(f32)
    p = (a * b).astype(f32)
    e = fma32(a, b, -p)
    exact = a.astype(np.float64) * b.astype(np.float64)
    assert np.array_equal(p.astype(np.float64) + e.astype(np.float64), exact)


def test_two_sum_is_error_free():
    rng = np.random.default_rng(2)
    x = (rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000)).astype(f32)
    y = (rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000)).astype(f32)
    s = (x + y).astype(f32)
    bv = (s - x).astype(f32)
    err = ((x - (s - bv)).astype(f32) + (y - bv).astype(f32)).astype(f32)
    assert np.array_equal(s.astype(np.float64) + err.astype(np.float64), x.astype(np.float64) + y.astype(np.float64))


def test_block_row_product_reaches_fp64_level_accuracy():
    rng = np.random.default_rng(3)
    b, nb, cols = 23, 30, 64
    # an on-site block of the DZP-like spectrum and couplings of the generator's scale
    H = [np.diag(rng.uniform(-25, 30, b))] + [0.5 * np.exp(-rng.uniform(0, 6.4)) * rng.standard_normal((b, b)) / np.sqrt(b)
                                              for _ in range(nb - 1)]
    V = [rng.standard_normal((b, cols)) * 1e-3 for _ in range(nb)]
    Hr = np.hstack(H)
    Vc = np.vstack(V)
    exact = Hr @ Vc
    got = pair_matmul(Hr, Vc)
    scale = np.abs(Hr) @ np.abs(Vc)          # the magnitude of the terms of each output
    rel = np.abs(got - exact) / scale
    assert np.median(rel) < 2.0 ** -43
    assert rel.max() < 2.0 ** -38
    f32_rel = np.abs((Hr.astype(f32) @ Vc.astype(f32)).astype(np.float64) - exact) / scale
    assert rel.max() < 1e-5 * f32_rel.max()
