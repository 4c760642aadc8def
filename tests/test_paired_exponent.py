"""Host model of the paired second-stage filter's exponent arithmetic (CPU only).

The kernel takes the colour dot product c'_p . c'_q (c' = c - 128) as one
dp4a of packed signed bytes started from the bit pattern of 1.5 * 2^23, reads
the result as a float f = 1.5 * 2^23 + c'_p . c'_q, and forms the exponent as
one FMA, f * 2kc + C_p with C_p = -kc |c'_p|^2 - 2kc * 1.5 * 2^23 rounded once
per pixel. The weights of one pixel then carry a common factor 2^(rounding of
C_p) that cancels in Eq. (1)'s quotient. This models each step in exact or
FP32 arithmetic and checks the claims: the packed bytes are c - 128, the biased
float is exact, and the normalised weights match the FP64 definition.
"""
import numpy as np

M = 12582912.0                  # 1.5 * 2^23
BIAS_BITS = 0x4B400000


def pack_centred(rgb):
    """Bytes r, g, b -> the packed word (r ^ 0x80) | (g ^ 0x80) << 8 | (b ^ 0x80) << 16."""
    r, g, b = (rgb[..., i].astype(np.uint32) for i in range(3))
    return (r | (g << 8) | (b << 16)) ^ np.uint32(0x00808080)


def dp4a_signed(a, b, c):
    """dp4a.s32.s32: c + sum of the four signed-byte products (two's complement wrap of int32)."""
    acc = c.astype(np.int64)
    for k in range(4):
        ai = ((a >> (8 * k)) & 0xFF).astype(np.int64)
        bi = ((b >> (8 * k)) & 0xFF).astype(np.int64)
        ai = np.where(ai >= 128, ai - 256, ai)
        bi = np.where(bi >= 128, bi - 256, bi)
        acc = acc + ai * bi
    return ((acc + 2 ** 31) % 2 ** 32 - 2 ** 31).astype(np.int64)


def fma32(a, b, c):
    """FP32 fused multiply-add: a * b + c exact in float64 here (48-bit product, aligned sum), one rounding."""
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(np.float32)


def test_packed_bytes_are_centred_colours():
    rgb = np.arange(256, dtype=np.uint8)[:, None].repeat(3, 1)
    w = pack_centred(rgb)
    for k in range(3):
        byte = ((w >> (8 * k)) & 0xFF).astype(np.int64)
        assert np.array_equal(np.where(byte >= 128, byte - 256, byte), np.arange(256) - 128)
    assert np.all((w >> 24) == 0)


def test_biased_dot_product_is_exact():
    rng = np.random.default_rng(3)
    p = rng.integers(0, 256, (20000, 3), dtype=np.uint8)
    q = rng.integers(0, 256, (20000, 3), dtype=np.uint8)
    # the extremes of the dot product: all 0 against all 0 (+3 * 128^2), 0 against 255 (-3 * 128 * 127)
    p[:2] = [[0, 0, 0], [0, 0, 0]]
    q[:2] = [[0, 0, 0], [255, 255, 255]]
    bits = dp4a_signed(pack_centred(p), pack_centred(q), np.full(len(p), BIAS_BITS, np.int64))
    f = bits.astype(np.uint32).view(np.float32).astype(np.float64)
    dot = ((p.astype(np.int64) - 128) * (q.astype(np.int64) - 128)).sum(1)
    assert np.array_equal(f - M, dot)
    assert dot.max() == 3 * 128 * 128 and dot.min() == -3 * 128 * 127


def test_weights_match_the_definition_after_normalisation():
    rng = np.random.default_rng(5)
    log2e = 1.4426950408889634
    for sigma_c in (17.5, 20.0, 40.0):
        kc = np.float32(log2e / (2.0 * sigma_c * sigma_c))
        kc2 = np.float32(2.0 * kc)
        bias = np.float32(-kc2 * np.float32(M))
        for _ in range(50):
            cp = rng.integers(0, 256, 3, dtype=np.uint8)
            cq = rng.integers(0, 256, (25, 3), dtype=np.uint8)
            # neighbours near the pixel's colour dominate the window, as in an image
            cq[:5] = np.clip(cp.astype(int) + rng.integers(-6, 7, (5, 3)), 0, 255)
            wp = pack_centred(cp[None])[0]
            n_p = int(((cp.astype(np.int64) - 128) ** 2).sum())
            c_p = fma32(-kc, np.float32(n_p), bias)                       # per pixel, rounded once
            f = dp4a_signed(np.full(25, wp, np.uint32), pack_centred(cq), np.full(25, BIAS_BITS, np.int64))
            f = f.astype(np.uint32).view(np.float32)
            e = fma32(f, kc2, c_p)                                          # per tap: one FMA
            n_q = ((cq.astype(np.int64) - 128) ** 2).sum(1)
            fq = np.exp2(-np.float64(kc) * n_q)                             # F_q
            w = np.exp2(e.astype(np.float64)) * fq
            exact = np.exp2(-np.float64(kc) * ((cq.astype(np.int64) - cp.astype(np.int64)) ** 2).sum(1))
            # FP32 rounding of an exponent up to kc 3 128^2 (about 88 at sigma_c 20): a few 2^-18
            assert np.allclose(w / w.sum(), exact / exact.sum(), rtol=1e-5, atol=1e-12)


def test_a_bias_rounded_per_tap_is_caught():
    """The normalisation check fails for the plausible slip the kernel avoids: folding a per-tap
    term (here the row part of the spatial exponent) into the biased constant, whose rounding at
    the bias's magnitude (about 2^-9) then differs from tap to tap and no longer cancels."""
    rng = np.random.default_rng(7)
    log2e = 1.4426950408889634
    kc = np.float32(log2e / (2.0 * 20.0 * 20.0))
    kc2 = np.float32(2.0 * kc)
    bias = np.float32(-kc2 * np.float32(M))
    worst = 0.0
    for _ in range(20):
        cp = rng.integers(0, 256, 3, dtype=np.uint8)
        cq = rng.integers(0, 256, (25, 3), dtype=np.uint8)
        cq[:5] = np.clip(cp.astype(int) + rng.integers(-6, 7, (5, 3)), 0, 255)
        n_p = int(((cp.astype(np.int64) - 128) ** 2).sum())
        c_p = fma32(-kc, np.float32(n_p), bias)
        f = dp4a_signed(np.full(25, pack_centred(cp[None])[0], np.uint32), pack_centred(cq),
                        np.full(25, BIAS_BITS, np.int64)).astype(np.uint32).view(np.float32)
        sy = np.float32(-0.0288) * np.float32(rng.integers(0, 3, 25) ** 2)     # -kp dy^2, sigma_p 5
        slip = fma32(f, kc2, (np.float64(c_p) + np.float64(sy)).astype(np.float32))
        n_q = ((cq.astype(np.int64) - 128) ** 2).sum(1)
        w = np.exp2(slip.astype(np.float64)) * np.exp2(-np.float64(kc) * n_q)
        exact = np.exp2(-np.float64(kc) * ((cq.astype(np.int64) - cp.astype(np.int64)) ** 2).sum(1) +
                        sy.astype(np.float64))
        a, b = w / w.sum(), exact / exact.sum()
        m = b > 1e-6
        worst = max(worst, float(np.max(np.abs(a[m] / b[m] - 1.0))))
    assert worst > 1e-4
