"""The split-TF32 product of the tensor-core kernel, emulated in numpy: x = hi + lo with hi = x with
its 13 low mantissa bits cleared and lo = x - hi; a TF32 MMA operand is read from its upper 19 bits
(truncation, as measured on the GPU).  The three-pass product lo_a hi_b + hi_a lo_b + hi_a hi_b
differs from the exact product by three terms, each below 2^-20 of it (the dropped lo_a lo_b, and
the truncation of lo_a and of lo_b to TF32), so by less than 3 * 2^-20 relative; the two-pass and
plain TF32 products are far less accurate; and fp16 / bf16 values (the 16-bit storage path) are
exact TF32 operands.
"""
import numpy as np


def tf32(x):
    """The value a TF32 MMA operand register holding FP32 x contributes (upper 19 bits)."""
    return (np.asarray(x, np.float32).view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def split(x):
    x = np.asarray(x, np.float32)
    hi = tf32(x)
    lo = (x - hi).astype(np.float32)  # exact in FP32
    return hi, lo


def test_split_is_exact_and_lo_is_small():
    x = np.random.default_rng(1).standard_normal(100000).astype(np.float32) * np.float32(7.0)
    hi, lo = split(x)
    assert np.array_equal(hi.astype(np.float64) + lo.astype(np.float64), x.astype(np.float64))
    nz = x != 0
    assert np.all(np.abs(lo[nz]) < np.abs(x[nz]) * 2.0 ** -10)
    assert np.array_equal(tf32(hi), hi)  # hi is itself a TF32 value


def test_three_pass_product_error_bound():
    g = np.random.default_rng(2)
    a = g.standard_normal(200000).astype(np.float32)
    b = g.standard_normal(200000).astype(np.float32)
    ah, al = split(a)
    bh, bl = split(b)
    f64 = lambda v: np.asarray(v, np.float64)
    exact = f64(a) * f64(b)
    # each MMA multiplies the operands' TF32 values exactly (11 x 11 significant bits)
    three = f64(tf32(al)) * f64(bh) + f64(ah) * f64(tf32(bl)) + f64(ah) * f64(bh)
    rel = np.abs(three - exact) / np.abs(exact)
    assert rel.max() < 3 * 2.0 ** -20
    two = f64(ah) * f64(bh) + f64(ah) * f64(tf32(bl))  # lo_a hi_b dropped
    assert (np.abs(two - exact) / np.abs(exact)).max() > 2.0 ** -12
    one = f64(ah) * f64(bh)  # plain TF32
    assert (np.abs(one - exact) / np.abs(exact)).max() > 2.0 ** -11


def test_gram_matrix_accuracy_of_the_split():
    """G = H^H H for a 32-antenna cluster block through the three-pass split, summed in FP64 here
    (the kernel accumulates in FP32): the split itself costs less than 1e-6 relative per entry."""
    g = np.random.default_rng(3)
    H = (g.standard_normal((16, 32)) + 1j * g.standard_normal((16, 32))).astype(np.complex64)
    re, im = H.real.astype(np.float32), H.imag.astype(np.float32)

    def prod3(x, y):
        xh, xl = split(x)
        yh, yl = split(y)
        f64 = lambda v: np.asarray(v, np.float64)
        return f64(tf32(xl)) @ f64(yh) + f64(xh) @ f64(tf32(yl)) + f64(xh) @ f64(yh)

    # Re G = Re^T Re + Im^T Im, Im G = Re^T Im - Im^T Re (G_uv = h_u^H h_v with rows h_u)
    G = (prod3(re, re.T) + prod3(im, im.T)) + 1j * (prod3(re, im.T) - prod3(im, re.T))
    Gx = np.conj(H.astype(np.complex128)) @ H.astype(np.complex128).T
    assert np.max(np.abs(G - Gx)) < 1e-6 * np.max(np.abs(Gx))


def test_16bit_values_are_exact_tf32_operands():
    g = np.random.default_rng(4)
    x16 = (g.standard_normal(100000) * 3).astype(np.float16)
    assert np.array_equal(tf32(x16.astype(np.float32)), x16.astype(np.float32))
    bf = (g.standard_normal(100000).astype(np.float32).view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32)
    assert np.array_equal(tf32(bf), bf)
    sub = np.array([6.0e-8, 1.0e-5, -3.0e-6], np.float16).astype(np.float32)  # fp16 subnormals
    assert np.array_equal(tf32(sub), sub)
