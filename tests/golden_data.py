"""Readers for the fixtures under tests/golden/: the paper's printed
coefficients and published reference values, each row with its citation."""
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


def air_viscosity_table():
    """(temperature K, dynamic viscosity N s/m^2) rows of the U.S. Standard
    Atmosphere 1976 fixture."""
    rows = []
    path = os.path.join(os.path.dirname(_PATH), "air_viscosity_us_standard_atmosphere_1976.txt")
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            _, T, mu = line.split()
            rows.append((float(T), float(mu)))
    return rows
