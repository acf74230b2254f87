"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake (a sign, an index, a swapped operand, a dropped
term, a wrong coefficient) in a copy of oracle/hx_oracle.c, builds it, and
runs the fast pins (tests/test_oracle_pins.py and the non-slow part of
tests/test_oracle_invariants.py) against that copy in a subprocess: every
copy must fail them.  The mistakes are planted on the CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hx_oracle.c")

MUTANTS = [
    ("d6 sign", "{0.0, 3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0}", "{0.0, 3.0 / 4.0, 3.0 / 20.0, 1.0 / 60.0}"),
    ("mid6 coefficient", "- 25.0 * f[-1]", "- 24.0 * f[-1]"),
    ("weno literal weights", "const double gam[3] = {1.0 / 16.0, 5.0 / 8.0, 5.0 / 16.0};\n    const double bet[3] = {b[0], b[1], b[2]};",
     "const double gam[3] = {5.0 / 16.0, 5.0 / 8.0, 1.0 / 16.0};\n    const double bet[3] = {b[0], b[1], b[2]};"),
    ("weno indicator order", "const double bet[3] = {b[0], b[1], b[2]};", "const double bet[3] = {b[2], b[1], b[0]};"),
    ("weno right candidate", "3.0 / 8.0 * W[4] - 5.0 / 4.0 * W[3] + 15.0 / 8.0 * W[2]",
     "3.0 / 8.0 * W[4] - 5.0 / 4.0 * W[3] + 15.0 / 8.0 * W[1]"),
    ("beta term", "b[1] = 13.0 / 12.0 * s2 * s2 + 1.0 / 4.0 * t2 * t2;", "b[1] = 13.0 / 12.0 * s2 * s2 + 1.0 / 4.0 * t2 * s2;"),
    ("eq19 coefficient", "13.0 / 320.0 * (f[2] - f[-2])", "13.0 / 230.0 * (f[2] - f[-2])"),
    ("eigenvector entry", "kx * (g - 1.0) * v / c2 + kz / rho", "kx * (g - 1.0) * v / c2 - kz / rho"),
    ("steger-warming energy", "(l4 + l5) * (3.0 - g) * s.c * s.c", "(l4 - l5) * (3.0 - g) * s.c * s.c"),
    ("node flux energy", "f[4] = (q[4] + s.p) * th;", "f[4] = (q[4] - s.p) * th;"),
    ("metric operand", "m[4] = prod_d(&C, CZ, ZETA, CX, XI, i, j, k)", "m[4] = prod_d(&C, CZ, ZETA, CY, XI, i, j, k)"),
    ("jacobian sign", "+ xz * yx * ze - xz * ye * zx", "+ xz * yx * ze + xz * ye * zx"),
    ("bulk viscosity", "const double lam = -2.0 / 3.0 * kv;", "const double lam = -1.0 / 3.0 * kv;"),
    ("heat-flux factor", "const double kq = kv / (P->pr * (P->gamma - 1.0));", "const double kq = kv / P->pr;"),
    ("rk3 stage 2", "3.0 / 4.0 * B->qn[t] + 1.0 / 4.0 * B->qs[t]", "1.0 / 4.0 * B->qn[t] + 3.0 / 4.0 * B->qs[t]"),
    ("chain rule without J", "J * (mx[0][c] * dc[v][0] + mx[1][c] * dc[v][1] + mx[2][c] * dc[v][2])",
     "(mx[0][c] * dc[v][0] + mx[1][c] * dc[v][1] + mx[2][c] * dc[v][2])"),
    ("residual sign", "B->r[c * N + p] = -J * B->r[c * N + p];", "B->r[c * N + p] = J * B->r[c * N + p];"),
    ("periodic translation", "for (int m = 0; m < 3; ++m) out[m] = c[m] + F->tr[m];",
     "for (int m = 0; m < 3; ++m) out[m] = c[m] - F->tr[m];"),
    ("closure stencil", "(-3.0 * f[0] + 4.0 * f[1] - f[2]) / 2.0", "(-3.0 * f[0] + 4.0 * f[1] + f[2]) / 2.0"),
    ("far-field invariant", "double Rm = unf - 2.0 * cinf / (g - 1.0);", "double Rm = unf + 2.0 * cinf / (g - 1.0);"),
    ("viscous flux row", "fv[2] = m[0] * txy + m[1] * tyy + m[2] * tyz;", "fv[2] = m[0] * txy + m[1] * tyy + m[2] * txz;"),
    ("interface tangential flip", "nid[p] = t > 0 ? id[a] : N->n[p] - 1 - id[a];", "nid[p] = id[a];"),
    ("interface layer", "nid[p] = nside ? N->n[p] - 1 - l : l;", "nid[p] = nside ? N->n[p] - l : l;"),
    ("local dt viscous factor", "(gp > 4.0 / 3.0 ? gp : 4.0 / 3.0)", "4.0 / 3.0"),
    ("local dt block", "const double h = dtl ? dtl[b][t % N] : dt[b];", "const double h = dtl ? dtl[0][t % N] : dt[b];"),
    ("face flux pairing", "qr[c] = UR[c * L + f + 1 + O];", "qr[c] = UR[c * L + f + O];"),
    ("wall node tangential velocity kept", "Qs[b][1 * N + p] = 0.0;", "(void)0;"),
    ("wall node normal velocity kept", "Qs[b][2 * N + p] = 0.0;", "(void)0;"),
    ("wall mirror tangential even", "        q[1] = -q[1];", "        q[1] = q[1];"),
    ("wall mirror normal even", "        q[2] = -q[2];", "        q[2] = q[2];"),
    ("far-field outgoing from free stream", "double Rp = uni + 2.0 * s.c / (g - 1.0);",
     "double Rp = unf + 2.0 * cinf / (g - 1.0);"),
    ("sutherland exponent", "return T * sqrt(T) * (1.0 + S) / (T + S);", "return T * (1.0 + S) / (T + S);"),
    ("sutherland sign of S", "return T * sqrt(T) * (1.0 + S) / (T + S);", "return T * sqrt(T) * (1.0 + S) / (T - S);"),
    ("sutherland normalisation", "return T * sqrt(T) * (1.0 + S) / (T + S);", "return T * sqrt(T) * S / (T + S);"),
    ("far-field entropy side", "    if (un > 0.0) {\n        ent = s.p", "    if (un < 0.0) {\n        ent = s.p"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation site not found: " + name
    c = tmp_path / "mutant.c"
    so = tmp_path / "mutant.so"
    c.write_text(src.replace(old, new, 1))
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99", "-fopenmp", "-o", str(so),
                    str(c), "-lm"], check=True, capture_output=True)
    env = dict(os.environ, HX_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m",
                        "not slow and not gpu", "tests/test_oracle_pins.py", "tests/test_oracle_invariants.py"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode != 0, "the pins did not catch: " + name
