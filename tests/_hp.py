"""High-precision (50-digit decimal) evaluation of the discrete H function,
independent of the oracle's log1p rearrangement."""
from decimal import Decimal, getcontext

getcontext().prec = 50


def H_dec(f, w):
    return sum(Decimal(float(a)) * (Decimal(float(a)) / Decimal(float(b))).ln() for a, b in zip(f, w))


def h_dec(f, d, w, alpha):
    """H(f + alpha d) - H(f) with every operation in 50-digit decimal."""
    A = Decimal(repr(alpha)) if isinstance(alpha, str) else Decimal(float(alpha))
    fn = [Decimal(float(a)) + A * Decimal(float(b)) for a, b in zip(f, d)]
    s = Decimal(0)
    for a, b in zip(fn, w):
        if a > 0:
            s += a * (a / Decimal(float(b))).ln()
    return s - H_dec(f, w)
