"""Property-based pins of the oracle's arithmetic (adversarial operands drawn by hypothesis,
checked against exact rationals): TwoSum / TwoProd exactness, the Joldes-Muller-Popescu bounds of
the accurate DW+DW, DW*DW, DW*FP, DW/FP and DW/DW, and the 2^-150 / 2^-200 bounds of the TD / QD
operations.  Skipped where hypothesis is not installed."""
from fractions import Fraction

import pytest

import oracle
from tests._exact import F, rel_err, split
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


_mag = st.floats(min_value=2.0 ** -200, max_value=2.0 ** 200)


@settings(max_examples=300, deadline=None)
@given(_mag, st.floats(-1, 1), _mag, st.booleans(), st.booleans())
def test_dd_by_binary64_property(x, fx, y, nx, ny):
    """DW*FP (Alg. 9, 2u^2) and DW/FP (Alg. 15, 3u^2) with a binary64 operand of any sign and an
    exponent up to 2^400 away."""
    a = _dw(-x if nx else x, fx)
    b = [-y if ny else y, 0.0]
    for op in ("mul_d", "div_d"):
        got = oracle.mp_op(op, 2, a, b)
        ex = _exact(op, a, b)
        assert rel_err(got, ex) <= BOUNDS_DD[op], (op, a, b, got)
        assert _norm_ok(got)


@settings(max_examples=300, deadline=None)
@given(_mag, st.floats(-1, 1), _mag, st.floats(-1, 1), st.booleans(), st.booleans())
def test_dd_div_property(x, fx, y, fy, nx, ny):
    """DW/DW (Alg. 17, 15u^2 + 56u^3) with both operands double-words."""
    a = _dw(-x if nx else x, fx)
    b = _dw(-y if ny else y, fy)
    got = oracle.mp_op("div", 2, a, b)
    assert rel_err(got, _exact("div", a, b)) <= BOUNDS_DD["div"], (a, b, got)
    assert _norm_ok(got)


def _mw(lead, fracs, w):
    """A w-component number: leading part `lead`, each lower part a fraction of the previous
    part's last bit (a normalised expansion with about 53w bits)."""
    c = [lead]
    for f in fracs[: w - 1]:
        c.append(c[-1] * f * 2.0 ** -53)
    return split(F(c), w)  # renormalised: the greedy w-component split of their exact sum


_fr = st.lists(st.floats(-1, 1), min_size=3, max_size=3)


@settings(max_examples=120, deadline=None)
@given(st.sampled_from([3, 4]), _mag, _fr, _mag, _fr, st.booleans(), st.booleans(),
       st.sampled_from(["add", "sub", "mul", "mul_d", "div", "div_d"]))
def test_td_qd_property(w, x, fx, y, fy, nx, ny, op):
    """TD / QD operations (exact evaluation, greedy rounding to w components) stay within
    2^-150 / 2^-200 of the exact result, on operands of any signs whose exponents differ by up to
    2^400; sums of nearly opposite numbers included (x + (-x)(1 + tiny))."""
    a = _mw(-x if nx else x, fx, w)
    b = _mw(-y if ny else y, fy, w)
    if op in ("mul_d", "div_d"):
        b = [b[0]] + [0.0] * (w - 1)
    bound = Fraction(2) ** (-150 if w == 3 else -200)
    got = oracle.mp_op(op, w, a, b)
    assert rel_err(got, _exact(op, a, b)) <= bound, (w, op, a, b, got)
    assert _norm_ok(got)
    if op in ("add", "sub"):  # heavy cancellation: b = -a (or a) perturbed in its last parts
        sgn = -1 if op == "add" else 1
        c = split(F(a) * sgn * (1 + Fraction(fy[0]) * Fraction(2) ** (-60 * w)), w)
        got = oracle.mp_op(op, w, a, c)
        ex = _exact(op, a, c)
        assert rel_err(got, ex) <= bound, (w, op, a, c, got)
