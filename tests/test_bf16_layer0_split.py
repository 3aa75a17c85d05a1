"""The BF16 engine's layer 0 runs as one K = 16 tensor-core op on BF16 high
and low parts: x = x_h + x_l, w = w_h + w_l (each part rounded to nearest
even), and the products x_h w_h + x_l w_h + x_h w_l plus b_h + b_l summed in
FP32; x_l w_l is dropped.  Checked here with BF16 rounding emulated in numpy:
the split represents an FP32 value to 2^-17 of it (the remainder after x_h is
at most 2^-8 of x and is itself rounded to 8 significant bits), the dropped
product is below 2^-16 of the term, and layer 0 so computed is within a few
2^-17 of the exact FP32 inputs' value -- far below the 2^-9 of the BF16
rounding its ReLU output then takes."""
import numpy as np


def bf16(x):
    """Round float32 to the nearest BF16 (ties to even), returned as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (r << 16).astype(np.uint32).view(np.float32)


def split2(x):
    x = np.asarray(x, dtype=np.float32)
    h = bf16(x)
    lo = bf16((x - h).astype(np.float32))  # x - h is exact in FP32
    return h, lo


def test_bf16_rounding_emulation():
    # exact BF16 values are fixed points; halfway cases go to even
    v = np.array([1.0, -2.5, 0.0, 3.0e-3], dtype=np.float32)
    v = bf16(v)
    assert np.array_equal(bf16(v), v)
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -7)  # BF16 spacing at 1
    assert bf16(one + ulp / 2) == one               # tie -> even (1.0)
    assert bf16(one + ulp + ulp / 2) == one + 2 * ulp  # tie -> even (1 + 2 ulp)
    assert bf16(one + ulp * 0.75) == one + ulp


def test_split_represents_fp32_to_2_pow_minus_17():
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, 200000).astype(np.float32)
    h, lo = split2(x)
    err = np.abs(x.astype(np.float64) - h.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -17 * np.abs(x.astype(np.float64)))
    # the low part is at most half a BF16 unit of the high part
    assert np.all(np.abs(lo) <= 2.0 ** -8 * np.abs(h) + 1e-30)


def test_layer0_split_sum_matches_fp32_layer0():
    rng = np.random.default_rng(11)
    n, W = 4096, 256
    p = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    w = (rng.standard_normal((W, 3)) / np.sqrt(3)).astype(np.float32)
    b = (0.01 * rng.standard_normal(W)).astype(np.float32)
    exact = p.astype(np.float64) @ w.astype(np.float64).T + b.astype(np.float64)
    ph, pl = split2(p)
    wh, wl = split2(w)
    bh, bl = split2(b)
    f = lambda a: a.astype(np.float64)
    split = (f(ph) @ f(wh).T + f(pl) @ f(wh).T + f(ph) @ f(wl).T) + (f(bh) + f(bl))
    dropped = f(pl) @ f(wl).T
    scale = np.abs(p.astype(np.float64)) @ np.abs(w.astype(np.float64)).T + np.abs(b.astype(np.float64))
    assert np.all(np.abs(dropped) <= 2.0 ** -16 * scale)
    # the representation errors of x and w (2^-17 each, relative) and the
    # dropped product bound the whole difference
    assert np.all(np.abs(split - exact) <= 2 * 2.0 ** -16 * scale + 1e-12)
    # far below the BF16 rounding of the layer's output (2^-9 relative)
    rel = np.abs(split - exact) / np.maximum(scale, 1e-30)
    assert rel.max() < 2.0 ** -14
