"""Property-based pins of the oracle's arithmetic (adversarial operands drawn by hypothesis,
checked against exact rationals): TwoSum / TwoProd exactness and the Joldes-Muller-Popescu bounds
of the accurate DW+DW and DW*DW.  Skipped where hypothesis is not installed."""
from fractions import Fraction

import pytest

import oracle
from tests._exact import rel_err
from tests.test_oracle_arith import BOUNDS_DD, _exact, _norm_ok

hyp = pytest.importorskip("hypothesis", reason="property tests need hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

_finite = st.floats(min_value=-2.0 ** 500, max_value=2.0 ** 500, allow_nan=False, allow_infinity=False,
                    allow_subnormal=False)


@settings(max_examples=400, deadline=None)
@given(_finite, _finite)
def test_eft_property(a, b):
    """TwoSum is exact for any pair whose sum does not overflow; TwoProd wherever the product's
    error term is representable (no underflow of a*b's low part, no overflow)."""
    s = oracle.two_sum(a, b)
    assert Fraction(s[0]) + Fraction(s[1]) == Fraction(a) + Fraction(b)
    if a != 0 and b != 0 and 2.0 ** -900 < abs(a * b) < 2.0 ** 900:
        p = oracle.two_prod(a, b)
        assert Fraction(p[0]) + Fraction(p[1]) == Fraction(a) * Fraction(b)


def _dw(hi, frac):
    """A normalised double-word hi + lo, lo a fraction of hi's last bit."""
    lo = hi * frac * 2.0 ** -53
    s = hi + lo
    return [s, (hi - s) + lo]


@settings(max_examples=300, deadline=None)
@given(st.floats(min_value=2.0 ** -200, max_value=2.0 ** 200), st.floats(-1, 1),
       st.floats(min_value=2.0 ** -200, max_value=2.0 ** 200), st.floats(-1, 1), st.booleans(), st.booleans())
def test_dd_add_mul_property(x, fx, y, fy, nx, ny):
    """Joldes-Muller-Popescu bounds for the accurate DW+DW (Alg. 6) and DW*DW (Alg. 12) on
    operands with independent signs and exponents up to 2^400 apart."""
    a = _dw(-x if nx else x, fx)
    b = _dw(-y if ny else y, fy)
    for op in ("add", "mul"):
        got = oracle.mp_op(op, 2, a, b)
        ex = _exact(op, a, b)
        assert rel_err(got, ex) <= BOUNDS_DD[op], (op, a, b, got)
        assert _norm_ok(got)
