"""Writes kde_weights_bw4.txt: g[d] = round(65536 exp(-d^2/(2 bw^2))) with
exp evaluated as an exact rational Taylor series (no floating point)."""
from fractions import Fraction


def exp_taylor(x: Fraction, terms: int = 80) -> Fraction:
    s, t = Fraction(0), Fraction(1)
    for n in range(terms):
        s += t
        t = t * x / (n + 1)
    return s


def weights(bw: int):
    out = []
    for d in range(3 * bw + 1):
        v = 65536 * exp_taylor(Fraction(-d * d, 2 * bw * bw))
        out.append(int((v + Fraction(1, 2)) // 1))
    return out


if __name__ == "__main__":
    print(" ".join(map(str, weights(4))))
