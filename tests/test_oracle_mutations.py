"""CPU: the oracles' pins catch plausible mistakes.  Each case copies the C
oracle into a temporary directory, plants one mistake in the copy (a
transposed or conjugated operand, a wrong phase, sign, factor, scale or
digit order), and runs that oracle's pin file against the copy in a child
process: some pins must fail while the rest still run.  The repository's own
oracle is never touched."""
import os
import re
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

# (pin file, C source, mistake, text in the source, replacement)
CASES = [
    ("test_oracle.py", "tpd_oracle.c", "transposed operand A[r][r^x]",
     "A[(r ^ x) * N + r]", "A[r * N + (r ^ x)]"),
    ("test_oracle.py", "tpd_oracle.c", "phase i^#Y instead of (-i)^#Y",
     "cplx w = times_minus_i_pow(acc, popc64(x & z));", "cplx w = times_minus_i_pow(acc, (4 - popc64(x & z)) & 3);"),
    ("test_oracle.py", "tpd_oracle.c", "conjugated weights",
     "  w.im = ldexp(w.im, -n);", "  w.im = -ldexp(w.im, -n);"),
    ("test_oracle.py", "tpd_oracle.c", "scale 2^(1-n) instead of 2^-n",
     "  w.re = ldexp(w.re, -n);\n  w.im = ldexp(w.im, -n);", "  w.re = ldexp(w.re, 1 - n);\n  w.im = ldexp(w.im, 1 - n);"),
    ("test_oracle.py", "tpd_alg2.c", "Alg. 2: Y as -i (a01 - a10) / 2",
     "W[i10].re = -((a01.im - a10.im) * 0.5); W[i10].im = (a01.re - a10.re) * 0.5;",
     "W[i10].re = (a01.im - a10.im) * 0.5; W[i10].im = -((a01.re - a10.re) * 0.5);"),
    ("test_oracle.py", "tpd_alg2.c", "Alg. 2: I computed as (a00 - a11) / 2",
     "W[i00].re = (a00.re + a11.re) * 0.5; W[i00].im = (a00.im + a11.im) * 0.5;",
     "W[i00].re = (a00.re - a11.re) * 0.5; W[i00].im = (a00.im - a11.im) * 0.5;"),
    ("test_oracle_weyl.py", "tpd_weyl.c", "omega^(+b.c) instead of omega^(-b.c)",
     "const int k = (d - ddot(b, c, d, n)) % d;", "const int k = ddot(b, c, d, n);"),
    ("test_oracle_weyl.py", "tpd_weyl.c", "transposed operand A[c][c+a]",
     "const wcplx x = A[dadd(c, a, d, n) * N + c];", "const wcplx x = A[c * N + dadd(c, a, d, n)];"),
    ("test_oracle_weyl.py", "tpd_weyl.c", "conjugated operand",
     "const wcplx x = A[dadd(c, a, d, n) * N + c];",
     "wcplx x = A[dadd(c, a, d, n) * N + c];\n        x.im = -x.im;"),
    ("test_oracle_weyl.py", "tpd_weyl.c", "scale d^-n left out",
     "const double scale = 1.0 / (double)N;", "const double scale = 1.0;"),
    ("test_oracle_gellmann.py", "tpd_gellmann.c", "antisymmetric element with the opposite sign",
     "    e[cnt++] = (gm_entry){c, r, 0.0, -1.0};\n    e[cnt++] = (gm_entry){r, c, 0.0, 1.0};",
     "    e[cnt++] = (gm_entry){c, r, 0.0, 1.0};\n    e[cnt++] = (gm_entry){r, c, 0.0, -1.0};"),
    ("test_oracle_gellmann.py", "tpd_gellmann.c", "transposed operand tr(G A^T)",
     "    const gcplx a = A[v * N + u];", "    const gcplx a = A[u * N + v];"),
    ("test_oracle_gellmann.py", "tpd_gellmann.c", "diagonal elements without their factor sqrt(2)",
     "const double f = sqrt(2.0 / ((double)l * (double)(l + 1)));",
     "const double f = sqrt(1.0 / ((double)l * (double)(l + 1)));"),
    ("test_oracle_gellmann.py", "tpd_gellmann.c", "qudit order reversed",
     "  for (int j = n - 1; j >= 0; --j) {", "  for (int j = 0; j < n; ++j) {"),
    ("test_oracle_gellmann.py", "tpd_gellmann.c", "identity's norm taken as 2",
     "    *norm = (double)d;", "    *norm = 2.0;"),
]


def _copy_tree(dst):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    os.makedirs(os.path.join(dst, "tests"))
    for f in os.listdir(HERE):
        if (f.startswith("test_oracle") and f.endswith(".py") and f != "test_oracle_mutations.py") or \
                f in ("conftest.py", "_helpers.py"):
            shutil.copy(os.path.join(HERE, f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(HERE, "golden"), os.path.join(dst, "tests", "golden"))
    pkg = os.path.join(dst, "paper_2310_13421_gb300")
    os.makedirs(pkg)
    open(os.path.join(pkg, "__init__.py"), "w").close()
    shutil.copy(os.path.join(ROOT, "paper_2310_13421_gb300", "synth.py"), pkg)


@pytest.mark.parametrize("pins,src,what,old,new", CASES, ids=[c[2] for c in CASES])
def test_planted_mistake_fails_pins(tmp_path, pins, src, what, old, new):
    _copy_tree(str(tmp_path))
    path = tmp_path / "oracle" / src
    text = path.read_text()
    assert old in text, "the mutation site moved: " + what
    path.write_text(text.replace(old, new))
    env = dict(os.environ, PYTHONPATH=str(tmp_path), OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", pins), "-q", "-p", "no:cacheprovider"],
                       cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    tail = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else r.stderr[-500:]
    failed = re.search(r"(\d+) failed", tail)
    passed = re.search(r"(\d+) passed", tail)
    assert failed and int(failed.group(1)) >= 1, "%s: no pin failed (%s)" % (what, tail)
    assert passed and int(passed.group(1)) >= 1, "%s: the pins did not run (%s)" % (what, tail)
