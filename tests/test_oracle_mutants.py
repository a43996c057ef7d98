"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
in a copy of rf_oracle.c (a dropped term, a wrong sign, a wrong coefficient
index, a transposed operand, the appendix's garbled constant, a lost
normalisation, swapped passes, a broken coast treatment), builds it, and
runs tests/test_oracle_pins.py against it: at least one pin must fail.
The copies live in oracle/_mutants/ (not part of the repository)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rf_oracle.c")
OUT = os.path.join(ROOT, "oracle", "_mutants")

MUTANTS = {
    "forward recursion drops its third term":
        ("if (i - j >= 0) v += alpha[3 * i + j - 1] * p[i - j];",
         "if (i - j >= 0 && j < 3) v += alpha[3 * i + j - 1] * p[i - j];"),
    "backward recursion takes the later point's coefficients":
        ("if (i + j < m) v += alpha[3 * i + j - 1] * x[i + j];",
         "if (i + j < m) v += alpha[3 * (i + j) + j - 1] * x[i + j];"),
    "backward sweep stops before the first point":
        ("for (int64_t i = m - 1; i >= 0; --i) {",
         "for (int64_t i = m - 1; i >= 1; --i) {"),
    "adjoint causal solve takes the current point's coefficients":
        ("if (r - j >= 0) v += alpha[3 * (r - j) + j - 1] * z[r - j];",
         "if (r - j >= 0) v += alpha[3 * r + j - 1] * z[r - j];"),
    "adjoint anticausal solve reads the wrong operand":
        ("if (r + j < m) v += alpha[3 * (r + j) + j - 1] * x[r + j];",
         "if (r + j < m) v += alpha[3 * (r + j) + j - 1] * z[r + j];"),
    "wrong sign of one Theorem 3.1 term":
        ("a[2] = -3.382473 * s2 - 3.000000 * s3;",
         "a[2] = 3.382473 * s2 - 3.000000 * s3;"),
    "the appendix's garbled P1":
        ("a[0] = 3.738128 + 5.788982 * s", "a[0] = 3.738128 + 5.788824 * s"),
    "beta without the Gaussian-peak factor":
        ("double g = (norm == 1) ? 1.0 : pow(2.0 * ORC_PI * sigma * sigma, 0.25);",
         "double g = 1.0;"),
    "Hayden's E without K":
        ("double E = (double)K / (sigma * sigma);", "double E = 1.0 / (sigma * sigma);"),
    "imaginary points rounded down":
        ("return (int64_t)ceil(img_factor * sigma_coast);",
         "return (int64_t)floor(img_factor * sigma_coast);"),
    "x and y passes swapped":
        ("int along_x = adjoint ? (pass == 1) : (pass == 0);",
         "int along_x = adjoint ? (pass == 0) : (pass == 1);"),
    "constant extension copies the far edge":
        ("for (int64_t r = 0; r < nl; ++r) w->x[r] = out[b];",
         "for (int64_t r = 0; r < nl; ++r) w->x[r] = out[b + L - 1];"),
    "constant extension without its transpose on the left":
        ("for (int64_t r = 0; r < nl; ++r) out[b] += w->x[r];", "(void)0;"),
    "q-correction solves the wrong quadratic":
        ("return 2.0 * s2 / (B + sqrt(B * B + 4.0 * A * s2));",
         "return 2.0 * s2 / (2.0 * B + sqrt(B * B + 4.0 * A * s2));"),
    "1st-RF normalisation per iteration instead of per pass":
        ("1.0 / (4.0 * (double)K));", "1.0 / (2.0 * (double)K));"),
    "1st-RF coefficient with the wrong root":
        ("*alpha = 1.0 + E - r;", "*alpha = 1.0 - E + r;"),
    "land output keeps the input":
        ("if (!mask[i]) { out[i] = 0.0; ++i; continue; }",
         "if (!mask[i]) { out[i] = in[i]; ++i; continue; }"),
    "left imaginary points take the right coast's length scale":
        ("int64_t src = r < nl ? 0 : (r >= nl + L ? L - 1 : r - nl);",
         "int64_t src = r < nl ? L - 1 : (r >= nl + L ? L - 1 : r - nl);"),
    "adjoint forgets the inner beta":
        ("for (int64_t r = 0; r < m; ++r) z[r] *= beta[r];", "(void)0;"),
    "carried coasts re-extend with zeros every iteration":
        ("if (coast != 2 || k == 0) {", "if (1) {"),
    "carried coasts in the forward operator only":
        ("if (coast != 2 || k == 0) {", "if (coast != 2 || k == 0 || adjoint) {"),
}


def run_pins_on(tag, source):
    """Build `source` as the oracle and run the pin tests against it;
    returns pytest's exit code and output."""
    os.makedirs(OUT, exist_ok=True)
    csrc = os.path.join(OUT, tag + ".c")
    with open(csrc, "w") as f:
        f.write(source)
    env = dict(os.environ, RF_ORACLE_SRC=csrc, RF_ORACLE_LIB=os.path.join(OUT, tag + ".so"))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-1500:] + r.stderr[-1500:]


def test_unmutated_copy_passes():
    """Control: the same build and run on an unchanged copy passes."""
    code, out = run_pins_on("control", open(SRC).read())
    assert code == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_the_planted_mistake(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not found once: {old}"
    code, out = run_pins_on("m%02d" % sorted(MUTANTS).index(name), src.replace(old, new))
    assert code == 1, (name, code, out)
