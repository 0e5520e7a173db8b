"""The arithmetic the FP64 tensor-core products rest on, restated on the host in NumPy:
rows scaled by a power of two with |x| < 2^e, 8 round-to-nearest slices of 7 bits, the 36
slice products with s + t < 8 accumulated per order s + t in FP32 over windows of 400 k and
combined in FP64.  Checked: the slice bounds (|d_0| <= 128, |d_s| <= 64), the remainder
(<= 2^-57 2^e), that every partial sum of an order stays below 2^24 (so FP32 holds it
exactly whatever its rounding: the FP32 running sums here equal the exact integer sums),
including an input that drives every slice to its largest magnitude, and the error of
the combined product against the exact one (K 2^-52 max|a_i| max|b_j|).  The device
kernel itself is tested on the GPU (tests/test_gpu_dgemm.py)."""
import numpy as np

S, BITS, WINDOW = 8, 7, 400


def slices(x):
    """Rows of x -> (d [S][rows][k] integer-valued float64, e [rows])."""
    m = np.abs(x).max(axis=1)
    e = np.where(m > 0, np.frexp(m)[1], 0)      # m = f 2^e with f in [1/2, 1): m < 2^e
    r = x / np.ldexp(1.0, e)[:, None]
    d = np.empty((S,) + x.shape)
    for s in range(S):
        t = r * 128.0
        d[s] = np.rint(t)
        r = t - d[s]
    return d, e, r


def product(a, b):
    da, ea, _ = slices(a)
    db, eb, _ = slices(b)
    k = a.shape[1]
    acc = np.zeros((a.shape[0], b.shape[0]))
    peak = 0.0
    for w0 in range(0, k, WINDOW):
        sl = slice(w0, min(k, w0 + WINDOW))
        for d in range(S):
            o32 = np.zeros((a.shape[0], b.shape[0]), np.float32)
            exact = np.zeros((a.shape[0], b.shape[0]))
            for s in range(d + 1):
                t = d - s
                for q in range(sl.start, sl.stop):        # one k at a time: every partial sum
                    p = np.outer(da[s][:, q], db[t][:, q])
                    exact += p
                    o32 += p.astype(np.float32)
                    peak = max(peak, float(np.abs(exact).max()))
            assert np.array_equal(o32.astype(np.float64), exact)   # FP32 held every partial sum
            acc += exact * 2.0 ** (-BITS * (d + 2))
    return acc * np.ldexp(1.0, ea)[:, None] * np.ldexp(1.0, eb)[None, :], peak


def test_slice_bounds_and_remainder():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((16, 257)) * 10.0 ** rng.uniform(-30, 30, size=(16, 1))
    x[2] = 0.0
    d, e, r = slices(x)
    assert np.all(d == np.rint(d))
    assert np.abs(d[0]).max() <= 128 and np.abs(d[1:]).max() <= 64
    recon = sum(d[s] * 2.0 ** (-BITS * (s + 1)) for s in range(S)) * np.ldexp(1.0, e)[:, None]
    assert np.all(np.abs(x - recon) <= 2.0 ** -57 * np.ldexp(1.0, e)[:, None])
    assert np.all(d[:, 2] == 0)


def test_order_sums_stay_exact_in_fp32_and_the_product_is_fp64_accurate():
    rng = np.random.default_rng(5)
    k = 900                                   # three windows, the last one partial
    a = rng.standard_normal((6, k)) * 10.0 ** rng.uniform(-20, 20, size=(6, 1))
    b = rng.standard_normal((5, k)) * 10.0 ** rng.uniform(-20, 20, size=(5, 1))
    c, peak = product(a, b)
    assert peak < 2.0 ** 24
    ref = a.astype(np.longdouble) @ b.astype(np.longdouble).T
    bound = k * 2.0 ** -52 * np.abs(a).max(axis=1)[:, None] * np.abs(b).max(axis=1)[None, :]
    assert np.all(np.abs(c.astype(np.longdouble) - ref) <= bound)


def test_largest_slices_stay_below_two_to_the_24():
    """Every slice at its largest magnitude with one sign: the worst case of the window."""
    per_k = sum((128 if s == 0 else 64) * (128 if d - s == 0 else 64) for d in range(S) for s in range(d + 1)
                if d == S - 1)
    worst = max(sum((128 if s == 0 else 64) * (128 if d - s == 0 else 64) for s in range(d + 1)) for d in range(S))
    assert worst == 2 * 128 * 64 + 6 * 64 * 64 == per_k
    assert worst * WINDOW < 2 ** 24 <= worst * (WINDOW + 10)
