"""The pins are pinned: each plausible mistake planted in a copy of the
oracle (a dropped factor, a wrong sign, a wrong index, a transposed operand,
a wrong unit, in the 3-D and 2-D steps, the sources, the Dirichlet nodes and
the adjoint) makes tests/test_oracle_pins.py fail.  The copy is compiled
like the oracle and loaded through BFVM_ORACLE_LIB in a child pytest run;
the oracle itself is untouched."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, text in oracle.c, replacement); the first occurrence is replaced
MUTANTS = [
    ("decay share not split over the three axes",
     "double ell = lambda[s] * dt / 3.0;", "double ell = lambda[s] * dt;"),
    ("line ends take the interior diagonal (no zero-flux face)",
     "diag[i] = 1.0 + ell + c * (double)(left + right);", "diag[i] = 1.0 + ell + c * 2.0;"),
    ("back substitution adds instead of subtracting",
     "x[i] = x[i] - cprime[i] * x[i + 1];", "x[i] = x[i] + cprime[i] * x[i + 1];"),
    ("lower diagonal tested on the wrong neighbour",
     "lower[i] = left ? -c : 0.0;", "lower[i] = right ? -c : 0.0;"),
    ("uptake dropped from the source denominator",
     "double b = w * (S[i * n_sub + s] + U[i * n_sub + s]);", "double b = w * S[i * n_sub + s];"),
    ("voxel volume taken as dx^2",
     "double v_vox = dx * dx * dx;", "double v_vox = dx * dx;"),
    ("explicit instead of implicit source update",
     "*r = (*r + a) / (1.0 + b);", "*r = *r + a - b * (*r);"),
    ("2-D variant: decay share of the 3-D step",
     "double ell = lambda[s] * dt / 2.0;", "double ell = lambda[s] * dt / 3.0;"),
    ("Dirichlet node holds half its value",
     "rho[(int64_t)sub[i] * n_vox + vox[i]] = val[i];",
     "rho[(int64_t)sub[i] * n_vox + vox[i]] = 0.5 * val[i];"),
    ("adjoint: sign of the diffusion gradient",
     "dD[s] -= (dt / (dx * dx))", "dD[s] += (dt / (dx * dx))"),
    ("adjoint: decay gradient without the LOD share",
     "dlambda[s] -= (dt / (double)dims)", "dlambda[s] -= dt"),
    ("adjoint: a node's entry is not zeroed",
     "for (int64_t i = 0; i < n_nodes; ++i) g[(int64_t)sub[i] * n_vox + vox[i]] = 0.0;",
     "for (int64_t i = 0; i < n_nodes; ++i) g[(int64_t)sub[i] * n_vox + vox[i]] *= 1.0;"),
]


def _compile(src_text, out_dir):
    c = os.path.join(out_dir, "oracle_mutant.c")
    so = os.path.join(out_dir, "liboracle_mutant.so")
    with open(c, "w") as f:
        f.write(src_text)
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", c,
            "-o", so, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return so


def _pins(lib):
    env = dict(os.environ, BFVM_ORACLE_LIB=lib)
    return subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", "test_oracle_pins.py"),
                           "-x", "-q", "-p", "no:cacheprovider"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmutated_copy_passes(tmp_path):
    """The harness itself: a faithful copy loaded the same way passes."""
    r = _pins(_compile(open(SRC).read(), str(tmp_path)))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, f"mutation site gone from oracle.c: {old!r}"
    r = _pins(_compile(src.replace(old, new, 1), str(tmp_path)))
    assert r.returncode != 0, f"the pins did not catch: {name}"
