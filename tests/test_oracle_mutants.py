"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy of the C
oracle (a wrong sign, a dropped term or factor, a swapped operand or index), builds it, and runs the pin
suites against it in a separate process, which must fail.  CPU only.

Transposing the orientation pair (o, i) of a tap is not among them: it is not a mistake for
these kernels.  The squared distances are even in the spatial offset and k(u^-1) = k(u), so
K_oi(d) = K_io(-d) = K_io(d) (pinned in test_taps_identity_and_symmetry)."""
import os
import subprocess
import sys

import pytest

from oracle import build as oracle_build
from oracle import lift as oracle_lift

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = [os.path.join(ROOT, "tests", "test_oracle_pins.py"), os.path.join(ROOT, "tests", "test_oracle_lift.py")]

# (name, exact text of the oracle source, its planted replacement)
MUTANTS = [
    ("half-angle sign", "double b1 = x * ch + y * sh;", "double b1 = x * ch - y * sh;"),
    ("rotation sign in the group product", "double x = a[0] + b[0] * ca - b[1] * sa;",
     "double x = a[0] + b[0] * ca + b[1] * sa;"),
    ("g h^-1 instead of h^-1 g", "or_group_mul(hi, g, u);\n    return -or_rho2",
     "or_group_mul(g, hi, u);\n    return -or_rho2"),
    ("dropped w2 term of rho_b",
     "return (w1 * b1) * (w1 * b1) + (w2 * b2) * (w2 * b2) + (w3 * b3) * (w3 * b3);",
     "return (w1 * b1) * (w1 * b1) + (w3 * b3) * (w3 * b3);"),
    ("flipped dy offset of the convolution", "int sy = y - dy, sx = x - dx;", "int sy = y + dy, sx = x - dx;"),
    ("transposed spatial offsets in the linear convolution",
     "acc += kt[((size_t)(o * nth + i) * D + (dy + r)) * D + (dx + r)] *",
     "acc += kt[((size_t)(o * nth + i) * D + (dx + r)) * D + (dy + r)] *"),
    ("x and y spacings swapped in the taps",
     "double g[3] = {(double)dx / nx, (double)dy / ny, 2.0 * OR_PI * o / nth};\n"
     "                    double h[3] = {0.0, 0.0, 2.0 * OR_PI * i / nth};\n"
     "                    lk[",
     "double g[3] = {(double)dx / ny, (double)dy / nx, 2.0 * OR_PI * o / nth};\n"
     "                    double h[3] = {0.0, 0.0, 2.0 * OR_PI * i / nth};\n"
     "                    lk["),
    ("sign of the w-update", "lwi[g] = lmu[(size_t)i * V + g] - lkv[g];", "lwi[g] = lmu[(size_t)i * V + g] + lkv[g];"),
    ("sign of the v-update", "lv[(size_t)i * V + g] += L[g] - ld[(size_t)i * V + g];",
     "lv[(size_t)i * V + g] += ld[(size_t)i * V + g] - L[g];"),
    ("uniform weights instead of lambda", "L[g] += lam[i] * ldi[g];", "L[g] += ldi[g] / n;"),
    ("sign in the logarithm of rho_c", "double c1 = (p * x + q * y) / det;", "double c1 = (p * x - q * y) / det;"),
    ("cost taps without 1/eps", "(c > 0.0 ? log(c) : -INFINITY) - c / eps;", "(c > 0.0 ? log(c) : -INFINITY) - c;"),
    ("second marginal of W2 from mu", "lb[g] = log(nu[g]) - t[g];", "lb[g] = log(mu[g]) - t[g];"),
    ("W2 dual without eps", "res[1] = eps * dual;", "res[1] = dual;"),
    ("prox constant without m", "double c = sigma * m / (m - 1.0), q = m - 1.0;",
     "double c = sigma / (m - 1.0), q = m - 1.0;"),
    ("sign of the JKO b-update", "lb[g] = u[g] - t[g];", "lb[g] = u[g] + t[g];"),
    ("marginal violation without the weights", "viol += lam[i] * s;", "viol += s;"),
    ("marginal violation not relative", "stats[1] = viol / mass;", "stats[1] = viol;"),
    ("log convolution without its shift", "    return M + log(acc);\n}", "    return log(acc);\n}"),
    ("log convolution skipping terms above double resolution", "if (t < -746.0) continue;",
     "if (t < -7.46) continue;"),
    ("log convolution shift over the first orientation only",
     "double M = -INFINITY;\n    for (int i = 0; i < nth; ++i)", "double M = -INFINITY;\n    for (int i = 0; i < 1; ++i)"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_a_planted_mistake(tmp_path, name, old, new):
    src = open(oracle_build.SRC).read()
    assert src.count(old) == 1, "the planted line no longer matches the oracle source: " + name
    mutant = tmp_path / "se2ot_oracle_mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libse2ot_oracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", str(mutant), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, SE2OT_ORACLE_LIB=str(lib))
    run = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + PINS,
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert run.returncode != 0, "no pin failed with the planted mistake: " + name
    assert "failed" in run.stdout, run.stdout[-2000:]


# the same for the lifting / projection oracle (Python): (name, exact text, planted replacement)
LIFT_MUTANTS = [
    ("lift bin by floor instead of rounding", "(2.0 * math.pi) + 0.5)) % nt", "(2.0 * math.pi))) % nt"),
    ("half the reconstruction angle", "th = 2.0 * math.pi * k / nt", "th = math.pi * k / nt"),
    ("negative part not negated", "up, um = np.maximum(U, 0.0), -np.minimum(U, 0.0)",
     "up, um = np.maximum(U, 0.0), np.minimum(U, 0.0)"),
    ("interpolated masses swapped", "b += sign * ((1.0 - t) * m0 + t * m1) * project(phi)",
     "b += sign * (t * m0 + (1.0 - t) * m1) * project(phi)"),
]


@pytest.mark.parametrize("name,old,new", LIFT_MUTANTS, ids=[m[0] for m in LIFT_MUTANTS])
def test_lift_pins_catch_a_planted_mistake(tmp_path, name, old, new):
    src = open(oracle_lift.__file__).read()
    assert src.count(old) == 1, "the planted line no longer matches the oracle source: " + name
    mutant = tmp_path / "lift_mutant.py"
    mutant.write_text(src.replace(old, new))
    env = dict(os.environ, SE2OT_ORACLE_LIFT=str(mutant))
    run = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", PINS[1]],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert run.returncode != 0, "no pin failed with the planted mistake: " + name
    assert "failed" in run.stdout, run.stdout[-2000:]
