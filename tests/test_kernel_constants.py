"""The rounded lattice constants of the collision kernel satisfy the
discrete moment identities exactly (checked in rational arithmetic from the
source), and each is representable in its type: mass and momentum of the
reconstruction are then conserved up to unbiased rounding."""
import os
import re
from fractions import Fraction

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_0707_1299_gb300", "csrc", "lb_device.cuh")


def _constants(typ):
    src = open(SRC).read()
    body = re.search(r"struct Wts<%s>\s*\{(.*?)\};" % typ, src, flags=re.S).group(1)
    vals = {}
    for name, m, e in re.findall(r"(\w+) = ([0-9.]+)f? \* 0x1p(-?\d+)f?;", body):
        vals[name] = Fraction(int(float(m))) * Fraction(2) ** int(e)
    for name, k, other in re.findall(r"(\w+) = ([0-9.]+)f? \* (w\d);", body):
        vals[name] = Fraction(int(float(k))) * vals[other]
    return vals


def test_weights_identities_exact():
    for typ, ctype in (("float", np.float32), ("double", np.float64)):
        c = _constants(typ)
        assert set(c) == {"w0", "w1", "w2", "a1", "b1"}
        assert c["w0"] + 6 * c["w1"] + 12 * c["w2"] == 1
        assert 2 * c["a1"] + 8 * c["b1"] == 1
        for v in c.values():
            assert Fraction(float(ctype(float(v)))) == v  # representable
        # and each is the nearest such value to the exact weight
        eps = np.finfo(ctype).eps
        for k, exact in (("w0", Fraction(1, 3)), ("w1", Fraction(1, 18)), ("w2", Fraction(1, 36)),
                         ("a1", Fraction(1, 6)), ("b1", Fraction(1, 12))):
            assert abs(c[k] / exact - 1) < 4 * eps
