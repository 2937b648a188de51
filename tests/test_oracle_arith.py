"""Pins for the oracle's multi-component arithmetic (Sec. 2 number formats).

Everything is checked against exact rational arithmetic (Python Fraction), never against the
oracle itself:
  * TwoSum / TwoProd are error-free: s + e == a + b and p + e == a * b exactly, plus closed-form
    cases from tests/golden/eft_cases.txt.
  * DD operations stay within the published bounds of Joldes, Muller, Popescu (TOMS 2017):
    Alg. 6 add 3u^2+13u^3, Alg. 9 DW*FP 2u^2, Alg. 12 DW*DW 5u^2, Alg. 15 DW/FP 3u^2,
    Alg. 17 DW/DW 15u^2+56u^3; square root: 4u^2 on the squared result.
  * TD / QD operations (exact evaluation, greedy rounding) stay within 2^-150 / 2^-200.
  * results are normalised: |c_{k+1}| <= 2^-52 |c_k|.
Operands include heavy cancellation (x + (-x + tiny)) and wide exponent gaps.
"""
import math
import os
import random
from fractions import Fraction

import pytest

import oracle
from tests._exact import F, U, rand_mp, rel_err, split

GOLD = os.path.join(os.path.dirname(__file__), "golden", "eft_cases.txt")


def _gold():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        op, a, b, hi, lo = line.split()
        rows.append((op, *(float.fromhex(v) for v in (a, b, hi, lo))))
    return rows


@pytest.mark.parametrize("row", _gold())
def test_eft_closed_forms(row):
    op, a, b, hi, lo = row
    got = oracle.two_sum(a, b) if op == "two_sum" else oracle.two_prod(a, b)
    assert got[0] == hi and got[1] == lo


def test_eft_exact_random():
    rng = random.Random(1)
    for _ in range(3000):
        a = rng.uniform(-1, 1) * 2.0 ** rng.randint(-60, 60)
        b = rng.uniform(-1, 1) * 2.0 ** rng.randint(-60, 60)
        s = oracle.two_sum(a, b)
        assert Fraction(s[0]) + Fraction(s[1]) == Fraction(a) + Fraction(b)
        assert s[0] == a + b
        p = oracle.two_prod(a, b)
        assert Fraction(p[0]) + Fraction(p[1]) == Fraction(a) * Fraction(b)


def _norm_ok(c):
    for k in range(len(c) - 1):
        if c[k] == 0:
            if any(x != 0 for x in c[k + 1:]):
                return False
            return True
        if abs(c[k + 1]) > abs(c[k]) * 2.0 ** -52 * (1 + 2.0 ** -50):
            return False
    return True


BOUNDS_DD = {"add": 3 * U ** 2 + 13 * U ** 3, "sub": 3 * U ** 2 + 13 * U ** 3, "mul_d": 2 * U ** 2,
             "mul": 5 * U ** 2, "div_d": 3 * U ** 2, "div": 15 * U ** 2 + 56 * U ** 3}


def _exact(op, a, b):
    A, B = F(a), F(b)
    if op == "add":
        return A + B
    if op == "sub":
        return A - B
    if op == "mul":
        return A * B
    if op == "mul_d":
        return A * Fraction(b[0])
    if op == "div":
        return A / B
    if op == "div_d":
        return A / Fraction(b[0])
    raise ValueError(op)


def _operands(rng, w, op, cancel):
    a = rand_mp(rng, w)
    if op in ("mul_d", "div_d"):
        b = [rand_mp(rng, 1)[0]] + [0.0] * (w - 1)
    else:
        b = rand_mp(rng, w)
    if cancel and op in ("add", "sub"):
        # b = -a (or +a for sub) perturbed far below a's leading bits: massive cancellation
        tiny = rand_mp(rng, w, emin=-110 * w, emax=-60)
        base = F(a) * (-1 if op == "add" else 1)
        b = split(base + F(tiny) * abs(F(a)), w)
    return a, b


@pytest.mark.parametrize("op", ["add", "sub", "mul_d", "mul", "div_d", "div"])
@pytest.mark.parametrize("cancel", [False, True])
def test_dd_bounds(op, cancel):
    rng = random.Random(hash((op, cancel)) & 0xFFFF)
    worst = Fraction(0)
    for _ in range(800):
        a, b = _operands(rng, 2, op, cancel)
        got = oracle.mp_op(op, 2, a, b)
        ex = _exact(op, a, b)
        e = rel_err(got, ex)
        worst = max(worst, e)
        assert e <= BOUNDS_DD[op], (op, a, b, got, float(e / U ** 2))
        assert _norm_ok(got)


def test_dd_sqrt():
    rng = random.Random(7)
    for _ in range(800):
        a = rand_mp(rng, 2, sign=1)
        s = oracle.mp_op("sqrt", 2, a)
        # relative error of s^2 against a is about twice that of s
        assert abs(F(s) ** 2 - F(a)) / F(a) <= 8 * U ** 2
        assert _norm_ok(s)


@pytest.mark.parametrize("w,bound_exp", [(3, -150), (4, -200)])
@pytest.mark.parametrize("op", ["add", "sub", "mul_d", "mul", "div_d", "div"])
def test_td_qd_bounds(w, bound_exp, op):
    rng = random.Random(w * 100 + len(op))
    bound = Fraction(2) ** bound_exp
    for cancel in (False, True):
        for _ in range(150):
            a, b = _operands(rng, w, op, cancel)
            got = oracle.mp_op(op, w, a, b)
            e = rel_err(got, _exact(op, a, b))
            assert e <= bound, (w, op, float(e) and math.log2(float(e)))
            assert _norm_ok(got)


@pytest.mark.parametrize("w,bound_exp", [(3, -148), (4, -198)])
def test_td_qd_sqrt(w, bound_exp):
    rng = random.Random(w)
    for _ in range(100):
        a = rand_mp(rng, w, sign=1)
        s = oracle.mp_op("sqrt", w, a)
        assert abs(F(s) ** 2 - F(a)) / F(a) <= Fraction(2) ** bound_exp


def test_d_is_plain_binary64():
    rng = random.Random(3)
    for _ in range(200):
        a, b = rng.uniform(-10, 10), rng.uniform(-10, 10)
        assert oracle.mp_op("add", 1, [a], [b])[0] == a + b
        assert oracle.mp_op("mul", 1, [a], [b])[0] == a * b
        assert oracle.mp_op("div", 1, [a], [b])[0] == a / b


def test_exact_results_are_exact():
    # 1/3 in QD: the exact quotient rounded greedily; 3 * (1/3)_QD misses 1 by < 2^-200
    q = oracle.mp_op("div", 4, [1.0, 0, 0, 0], [3.0, 0, 0, 0])
    assert abs(F(q) * 3 - 1) < Fraction(2) ** -200
    # x + (-x) == 0 exactly for every w
    for w in (1, 2, 3, 4):
        x = rand_mp(random.Random(w), w)
        assert all(c == 0 for c in oracle.mp_op("sub", w, x, x))

