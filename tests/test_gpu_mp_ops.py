"""The library's multi-component arithmetic on the device (mpk_mp_op) against exact rationals.

Bounds (relative to the exact result, cancellation included), u = 2^-53:
  * D: correctly rounded (u);
  * DD: the published bounds of Joldes, Muller and Popescu (TOMS 2017) for the algorithms used:
    DW+DW 3u^2 + 13u^3, DW*FP 2u^2, DW*DW 5u^2, DW/FP 3u^2, DW/DW 15u^2 + 56u^3; the square root
    (one Newton correction of the binary64 root) 4u^2;
  * TD, QD: 2^-155 and 2^-208 (the renormalisation keeps about 53 w bits; measured 2^-159 /
    2^-213 on these operand families).
Operands: random numbers with about 53 w significant bits and exponents in [-250, 250], pairs that
cancel to a random depth, entries with zero lower components, and entries whose last component
sits at the bottom of the format.
"""
import random
from fractions import Fraction

import numpy as np
import pytest
import torch

from _exact import F, rand_mp, split
from paper_2504_14498_gb300 import _lib

pytestmark = pytest.mark.gpu

U = Fraction(1, 2 ** 53)
BOUND = {
    1: {op: U for op in ("add", "sub", "mul", "mul_fp", "div", "div_fp", "sqrt")},
    2: {"add": 3 * U ** 2 + 13 * U ** 3, "sub": 3 * U ** 2 + 13 * U ** 3, "mul": 5 * U ** 2, "mul_fp": 2 * U ** 2,
        "div": 15 * U ** 2 + 56 * U ** 3, "div_fp": 3 * U ** 2, "sqrt": 4 * U ** 2},
    3: {op: Fraction(1, 2 ** 155) for op in ("add", "sub", "mul", "mul_fp", "div", "div_fp", "sqrt")},
    4: {op: Fraction(1, 2 ** 208) for op in ("add", "sub", "mul", "mul_fp", "div", "div_fp", "sqrt")},
}
N = 1500


def _operands(w, seed):
    rng = random.Random(seed)
    A, B = [], []
    for t in range(N):
        a = rand_mp(rng, w, -250, 250)
        b = rand_mp(rng, w, -250, 250)
        kind = t % 4
        if kind == 1:  # cancellation: b = -a (1 + small)
            b = split(-F(a) * (1 + Fraction(rng.randint(-2 ** 20, 2 ** 20), 2 ** rng.randint(20, 53 * w + 10))), w)
        elif kind == 2:  # zero lower components
            a = [a[0]] + [0.0] * (w - 1)
        elif kind == 3 and w > 1:  # last component at the bottom of the format
            b = [b[0]] + [0.0] * (w - 2) + [b[0] * 2.0 ** (-53 * w + 3)]
        A.append(a)
        B.append(b)
    return np.array(A, dtype=np.float64).ravel(), np.array(B, dtype=np.float64).ravel()


def _exact(op, a, b):
    if op == "add":
        return a + b
    if op == "sub":
        return a - b
    if op == "mul":
        return a * b
    if op == "div":
        return a / b
    raise ValueError(op)


@pytest.mark.parametrize("w", [1, 2, 3, 4])
@pytest.mark.parametrize("op", ["add", "sub", "mul", "mul_fp", "div", "div_fp", "sqrt"])
def test_op_within_bound(w, op):
    a, b = _operands(w, 1000 * w + len(op))
    if op == "sqrt":
        A = a.reshape(-1, w)
        a = (A * np.sign(A[:, :1])).ravel()  # every entry negated where negative: positive values
    got = _lib.mp_op(op, w, torch.as_tensor(a, device="cuda"), torch.as_tensor(b, device="cuda")).cpu().numpy()
    bound = BOUND[w][op]
    worst = Fraction(0)
    for i in range(N):
        x = F(a[i * w:(i + 1) * w])
        y = F(b[i * w:(i + 1) * w])
        z = F(got[i * w:(i + 1) * w])
        if op == "mul_fp":
            ex = x * Fraction(float(b[i * w]))
        elif op == "div_fp":
            ex = x / Fraction(float(b[i * w]))
        elif op == "sqrt":
            # exact check without a square root: |z^2 - x| <= 2 bound x (1 + bound) covers |z - sqrt x| <= bound sqrt x
            err = abs(z * z - x) / x
            worst = max(worst, err / 2)
            assert err <= 2 * bound * (1 + bound) * 1.01, (i, float(err))
            continue
        else:
            ex = _exact(op, x, y)
        if ex == 0:
            assert z == 0, i
            continue
        rel = abs(z - ex) / abs(ex)
        worst = max(worst, rel)
        assert rel <= bound, (op, w, i, float(rel), float(bound))
    print(op, w, "worst relative error 2^%.1f" % (np.log2(float(worst)) if worst > 0 else -9999))


@pytest.mark.parametrize("w", [3, 4])
def test_components_normalised(w):
    """Results have decreasing component magnitudes, each within about an ulp of the one before
    (the top-down renormalisation can leave a component slightly above half an ulp of its
    predecessor), so the leading part approximates the value."""
    a, b = _operands(w, 77 + w)
    got = _lib.mp_op("mul", w, torch.as_tensor(a, device="cuda"), torch.as_tensor(b, device="cuda")).cpu().numpy()
    g = got.reshape(-1, w)
    for r in g:
        for k in range(1, w):
            if r[k] != 0.0:
                assert abs(r[k]) <= 2 * np.spacing(abs(r[k - 1])), r


def test_exact_cancellation_and_zero():
    for w in (1, 2, 3, 4):
        a, _ = _operands(w, 5)
        got = _lib.mp_op("sub", w, torch.as_tensor(a, device="cuda"), torch.as_tensor(a, device="cuda")).cpu().numpy()
        assert np.all(got == 0.0)
