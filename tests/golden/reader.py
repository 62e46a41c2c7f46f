"""Reader for the hand-worked fixtures in tests/golden (fractions allowed)."""
import os
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    out = {}
    with open(os.path.join(HERE, name)) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    i = 0
    n = None
    while i < len(lines):
        tok = lines[i].split()
        key = tok[0]
        if key == "n":
            n = int(tok[1])
            i += 1
        elif len(tok) == 1:
            rows = [[Fraction(v) for v in lines[i + 1 + r].split()] for r in range(n)]
            out[key] = rows
            i += 1 + n
        else:
            out[key] = [Fraction(v) for v in tok[1:]]
            i += 1
    out["n"] = n
    return out
