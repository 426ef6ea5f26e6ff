"""The forward splat's FP32-pipe cosine (cos_poly2 in csrc/gws_splat.cu, used by the tile
configurations that move part of the MUFU's load onto the FMA pipe): its coefficients, read from
the source, evaluated in float32 as the kernel does (nearest-turn reduction with a two-part 2 pi,
Horner in r^2), against the FP64 cosine over the arguments the kernel gives it (a few turns
around zero)."""
import math
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2505_06582_gb300", "csrc",
                   "gws_splat.cu")


def _constants():
    body = open(SRC).read().split("float2 cos_poly2(float2 x) {", 1)[1].split("\n}\n", 1)[0]
    return [np.float32(float(v)) for v in re.findall(r"pair\(([-0-9.e]+)f\)", body)]


def _cos_poly_f32(x):
    c = _constants()
    inv2pi, magic, neg_magic, m2pi_hi, m2pi_lo = c[0], c[1], c[2], c[3], c[4]
    coef = c[5:]  # Horner order: c6, c5 (first FMA), then c4 .. c0
    f32 = np.float32
    # FMA = one rounding: evaluate the product-sum in float64, round once (exact for these magnitudes)
    fma = lambda a, b, d: (a.astype(np.float64) * b + d).astype(f32)
    k = (fma(x, inv2pi, magic) + neg_magic).astype(f32)
    r = fma(k, m2pi_hi, x)
    r = fma(k, m2pi_lo, r)
    t = (r * r).astype(f32)
    p = fma(t, coef[0], coef[1])
    for ck in coef[2:]:
        p = fma(p, t, ck)
    return p


def test_cos_poly_error_bound_over_the_kernel_arguments():
    x = np.linspace(-25.0, 25.0, 2_000_001).astype(np.float32)
    err = np.abs(_cos_poly_f32(x).astype(np.float64) - np.cos(x.astype(np.float64)))
    assert err.max() < 5e-7, err.max()


def test_cos_poly_constants_are_the_reduction_and_a_degree_12_fit():
    c = _constants()
    assert abs(c[0] - 1 / (2 * math.pi)) < 1e-8 and c[1] == 12582912.0 and c[2] == -12582912.0
    assert abs(-c[3] - np.float32(2 * math.pi)) == 0 and abs(-c[3] - c[4] - 2 * math.pi) < 1e-12
    assert len(c) == 5 + 7  # seven even coefficients
