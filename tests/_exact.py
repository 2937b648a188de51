"""Exact rational helpers for the oracle pins (Python Fraction; no oracle code)."""
import random
from fractions import Fraction

U = Fraction(1, 2 ** 53)


def F(comps):
    return sum((Fraction(float(c)) for c in comps), Fraction(0))


def split(v, w):
    """Greedy w-component binary64 split of a rational (float(Fraction) rounds to nearest)."""
    out = []
    for _ in range(w):
        f = float(v)
        out.append(f)
        v -= Fraction(f)
    return out


def rand_mp(rng: random.Random, w, emin=-30, emax=30, sign=None):
    """Random w-component number with about 53w significant bits."""
    e = rng.randint(emin, emax)
    m = rng.getrandbits(53 * w + 8) | (1 << (53 * w + 7))
    v = Fraction(m, 1 << (53 * w + 7)) * Fraction(2) ** e
    if (sign is None and rng.random() < 0.5) or sign == -1:
        v = -v
    return split(v, w)


def rel_err(got, exact):
    if exact == 0:
        return Fraction(0) if F(got) == 0 else Fraction(10 ** 9)
    return abs(F(got) - exact) / abs(exact)
