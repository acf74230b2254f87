"""Reader for tests/golden/paper_coefficients.txt (paper-printed constants)."""
import os
from fractions import Fraction

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_coefficients.txt")


def coefficients():
    out = {}
    with open(_PATH) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            name, idx, val = line.split()
            out.setdefault(name, {})[int(idx)] = Fraction(val)
    return out
