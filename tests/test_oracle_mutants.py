"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a dropped
term, an off-by-one degree of freedom, a transposed operand, a flipped sign,
a missing factor, a wrong weight, a wrong generator constant, swapped
normals, a truncated acceptance test, uncentred ratings, reversed ties),
builds it with gcc on the CPU and runs the oracle's pin tests against that
build in a fresh interpreter: at least one pin must fail.  Nothing here
touches a GPU or the CUDA library.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "bpmf_oracle.c")

MUTANTS = {
    # W*^-1 without the prior-mean term beta0 n / (beta0 + n) (mu0 - xbar)(mu0 - xbar)^T
    "drop_nw_term": ("w * (mu0[a] - xbar[a]) * (mu0[b] - xbar[b])", "0.0 * (mu0[a] - xbar[a])"),
    # Bartlett diagonal k with nu - k + 1 degrees of freedom instead of nu - k
    "bartlett_dof": ("0.5 * (nu - (double)k)", "0.5 * (nu - (double)k + 1.0)"),
    # back substitution with L instead of L^T
    "row_transpose": ("t -= L[k * K + i] * x[k];", "t -= L[i * K + k] * x[k];"),
    # rating term of the right-hand side with the wrong sign
    "rhs_sign": ("b[a] += alpha * r[e] * v[a];", "b[a] -= alpha * r[e] * v[a];"),
    # precision without the noise precision alpha
    "drop_alpha": ("P[a * K + c] += alpha * v[a] * v[c];", "P[a * K + c] += v[a] * v[c];"),
    # posterior mean weighting the sample mean by 1 instead of n
    "mu_star_weight": ("(beta0 * mu0[a] + dn * xbar[a])", "(beta0 * mu0[a] + xbar[a])"),
    # a Philox round constant off by one
    "philox_constant": ("(uint64_t)0xD2511F53u * (uint64_t)x0", "(uint64_t)0xD2511F55u * (uint64_t)x0"),
    # Box-Muller with the sine and cosine normals swapped
    "box_muller_swap": ("*z0 = r * cos(2.0 * pi * u2);", "*z0 = r * sin(2.0 * pi * u2);"),
    # Gamma acceptance without the log(v) term
    "gamma_accept": ("+ d - d * v + d * log(v))", "+ d - d * v)"),
    # ratings not centred by the training mean
    "no_centring": ("cval[p] = (double)val[e] - mean;", "cval[p] = (double)val[e];"),
    # degree ties broken by descending row id
    "degree_ties": ("return a < b ? -1 : (a > b ? 1 : 0);", "return a > b ? -1 : (a < b ? 1 : 0);"),
}

RUNNER = r"""
import os, sys
sys.path.insert(0, {root!r}); sys.path.insert(0, os.path.join({root!r}, "tests"))
import oracle
oracle._SRC = {src!r}
oracle._LIB = {lib!r}
import pytest
sys.exit(pytest.main(["-q", "-x", "--no-header", "-p", "no:cacheprovider",
                      os.path.join({root!r}, "tests", "test_oracle_rng.py"),
                      os.path.join({root!r}, "tests", "test_oracle_hyper.py"),
                      os.path.join({root!r}, "tests", "test_oracle_row.py"),
                      os.path.join({root!r}, "tests", "test_oracle_structure.py")]))
"""


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_a_pin(tmp_path, name):
    good, bad = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(good) == 1, name
    msrc = tmp_path / "bpmf_oracle.c"
    msrc.write_text(src.replace(good, bad))
    mlib = tmp_path / "libbpmf_oracle.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
                    "-ffp-contract=off", "-o", str(mlib), str(msrc), "-lm"], check=True)
    code = RUNNER.format(root=ROOT, src=str(msrc), lib=str(mlib))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900,
                       cwd=str(tmp_path))
    assert r.returncode != 0, f"no pin caught {name}:\n{r.stdout[-1500:]}"


def test_unmodified_source_passes_the_same_runner(tmp_path):
    """The control: the runner itself passes on the oracle as written, so a
    mutant's failure comes from the planted mistake."""
    msrc = tmp_path / "bpmf_oracle.c"
    msrc.write_text(open(SRC).read())
    mlib = tmp_path / "libbpmf_oracle.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
                    "-ffp-contract=off", "-o", str(mlib), str(msrc), "-lm"], check=True)
    code = RUNNER.format(root=ROOT, src=str(msrc), lib=str(mlib))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900,
                       cwd=str(tmp_path))
    assert r.returncode == 0, r.stdout[-1500:]
