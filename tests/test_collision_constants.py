"""The FP32 constants of the collision conserve the density and momentum
deviations exactly in the update's linear part (Section 2, Eq. 2-3: the
collision keeps rho and rho u).  Read from the device header and checked in
exact rational arithmetic:

* the weights sum to exactly 1 (the factor on the density deviation per
  step is om1 + om * sum W, which is then 1 because om + om1 == 1);
* T = 2 (W1 + 2 W5) equals the header's double constant, and the force scale
  is 1 / (2 T) to double rounding;
* each weight is within 1e-7 of the printed one (Section 2).

With the weights rounded one by one the sum is 1 + 7.5e-9, and together with
1 - 1/tau rounded apart from 1/tau the deviations grew or shrank by up to
0.3 % over 40,000 steps; the GPU decay-run parity tests detect that."""
import os
import re
from fractions import Fraction as Q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_0707_2437_gb300", "csrc", "lbm_device.cuh")


def _hexconst(name):
    src = open(HDR).read()
    m = re.search(r"#define\s+" + name + r"\s+(0x[0-9a-fA-F.]+p[+-]?\d+)f?\b", src)
    assert m, name
    return Q(float.fromhex(m.group(1)))


def test_weights_sum_to_one_exactly_and_match_the_paper():
    w0, w1, w5 = _hexconst("VSS_W0"), _hexconst("VSS_W1"), _hexconst("VSS_W5")
    assert w0 + 4 * w1 + 4 * w5 == 1
    for w, printed in ((w0, Q(4, 9)), (w1, Q(1, 9)), (w5, Q(1, 36))):
        assert abs(w / printed - 1) < Q(1, 10 ** 7)
        # representable in FP32: 24 significant bits
        num, den = w.numerator, w.denominator
        assert den & (den - 1) == 0 and num.bit_length() <= 24


def test_momentum_and_force_constants_follow_the_weights():
    w1, w5 = _hexconst("VSS_W1"), _hexconst("VSS_W5")
    T = 2 * (w1 + 2 * w5)
    assert _hexconst("VSS_T_D") == T
    scale = _hexconst("VSS_A15_SCALE_D")
    assert abs(scale * 2 * T - 1) < Q(1, 2 ** 52)
