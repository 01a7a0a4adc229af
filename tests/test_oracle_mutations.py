"""The oracle's pins catch plausible mistakes: each mutant below is a copy of the
oracle's C source with one mistake planted (a dropped term, a wrong index or bound, a
wrong tie rule, a wrong compensation sign), compiled on the side and run against the
pins of ``test_oracle_pins.py`` in a child process. Every mutant must make some pin
fail; the unmutated copy, built and loaded the same way, must pass them all."""
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "spd_oracle.c")

# (what the mistake is, text in the source, its replacement: the first occurrence only)
MUTANTS = [
    ("row split drops the remainder", "bounds[c] = (c * n) / P;", "bounds[c] = (c * (n - 1)) / P;"),
    ("merge path takes a nonzero before a finished row's end",
     "if (r < n && pos[r + 1] <= p) {", "if (r < n && pos[r + 1] < p) {"),
    ("position split keeps a row that ends at the position",
     "while (r < n && pos[r + 1] <= q) ++r;", "while (r < n && pos[r + 1] < q) ++r;"),
    ("SpMV gathers x at the row index", "acc += vals[jB] * x[j];", "acc += vals[jB] * x[i];"),
    ("TwoSum adds its second error term with the wrong sign",
     "*e = (a - (x - z)) + (b - z);", "*e = (a - (x - z)) - (b - z);"),
    ("TwoProduct drops the product's rounding error", "*e = fma(a, b, -x);", "*e = 0.0;"),
    ("the triple product drops its second-order term",
     "cs->lo += q + (e2 + e * c);", "cs->lo += q + e2;"),
    ("SpMM gathers the row of X at the output row",
     "for (int64_t l = 0; l < L; ++l) yr[l] += vals[p] * X[j * ldx + l];",
     "for (int64_t l = 0; l < L; ++l) yr[l] += vals[p] * X[(i % (j + 1)) * ldx + l];"),
    ("SpMM^T overwrites instead of accumulating",
     "for (int64_t l = 0; l < L; ++l) dX[j * ldx + l] += vals[p] * dY[i * ldy + l];",
     "for (int64_t l = 0; l < L; ++l) dX[j * ldx + l] = vals[p] * dY[i * ldy + l];"),
    ("SDDMM drops the sampled value B(i,j)",
     "for (int64_t k = 0; k < K; ++k) acc += (b * C[i * ldc + k]) * Dnk[j * ldd + k];",
     "for (int64_t k = 0; k < K; ++k) acc += C[i * ldc + k] * Dnk[j * ldd + k];"),
    ("compensated SDDMM finds the wrong row at a row boundary",
     "else while (pos[i + 1] <= p) ++i;", "else while (pos[i + 1] < p) ++i;"),
    ("SpTTV keeps only the last product of a fiber",
     "for (int64_t p = pos2[f]; p < pos2[f + 1]; ++p) acc += vals[p] * c[crd2[p]];",
     "for (int64_t p = pos2[f]; p < pos2[f + 1]; ++p) acc = vals[p] * c[crd2[p]];"),
    ("SpMTTKRP drops the factor C(j,l)",
     "for (int64_t l = 0; l < R; ++l) ar[l] += (vals[p] * C[j * ldc + l]) * D[k * ldd + l];",
     "for (int64_t l = 0; l < R; ++l) ar[l] += vals[p] * D[k * ldd + l];"),
    ("validation accepts a final pos below the child count",
     "if (pos[nparent] != ncrd)", "if (pos[nparent] > ncrd)"),
    ("transpose records the column instead of the row", "t_crd[q] = (int32_t)i;", "t_crd[q] = (int32_t)crd[p];"),
    ("transpose records the output slot instead of A's position", "perm[q] = (int32_t)p;", "perm[q] = (int32_t)q;"),
    ("SpAdd3 drops B + C where D also stores the coordinate",
     "v = have ? v + t : t; ++pd;", "v = t; ++pd;"),
    ("column blocks take an inclusive upper bound",
     "crd[p] < bounds[b + 1]", "crd[p] <= bounds[b + 1]"),
    ("compensated SpMV returns only its leading part",
     "csum_add_prod(&acc, vals[jB], x[crd[jB]]);\n        y[t] = csum_value(&acc);",
     "csum_add_prod(&acc, vals[jB], x[crd[jB]]);\n        y[t] = acc.hi;"),
    ("compensated SpMM returns only its leading part",
     "for (int64_t l = 0; l < L; ++l) Y[t * ldy + l] = csum_value(&acc[l]);",
     "for (int64_t l = 0; l < L; ++l) Y[t * ldy + l] = acc[l].hi;"),
    ("compensated SpMM^T drops the final fold of its low parts",
     "for (int64_t l = 0; l < L; ++l) dX[j * ldx + l] += lo[j * L + l];",
     "for (int64_t l = 0; l < L; ++l) dX[j * ldx + l] += 0.0 * lo[j * L + l];"),
    ("compensated SDDMM drops the rounding error of B*C",
     "csum_add_prod3(&acc, b, C[i * ldc + k], Dnk[j * ldd + k]);",
     "csum_add_prod(&acc, b * C[i * ldc + k], Dnk[j * ldd + k]);"),
    ("compensated SDDMM returns only its leading part",
     "csum_add_prod3(&acc, b, C[i * ldc + k], Dnk[j * ldd + k]);\n        out[t] = csum_value(&acc);",
     "csum_add_prod3(&acc, b, C[i * ldc + k], Dnk[j * ldd + k]);\n        out[t] = acc.hi;"),
    ("compensated SpTTV returns only its leading part",
     "csum_add_prod(&acc, vals[p], c[crd2[p]]);\n        out[t] = csum_value(&acc);",
     "csum_add_prod(&acc, vals[p], c[crd2[p]]);\n        out[t] = acc.hi;"),
    ("compensated SpMTTKRP returns only its leading part",
     "for (int64_t l = 0; l < R; ++l) A[t * lda + l] = csum_value(&acc[l]);",
     "for (int64_t l = 0; l < R; ++l) A[t * lda + l] = acc[l].hi;"),
]


def _compile(src_text, outdir, name):
    c = os.path.join(outdir, name + ".c")
    so = os.path.join(outdir, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call([os.environ.get("CC", "gcc"), *oracle.CFLAGS, "-o", so, c, "-lm"])
    return so


def _pins_pass(lib_path):
    env = dict(os.environ, SPD_ORACLE_LIB=lib_path)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x",
                        "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    return r.returncode == 0, r.stdout[-2000:]


def test_every_planted_mistake_fails_a_pin():
    with open(SRC) as f:
        src = f.read()
    for what, a, b in MUTANTS:
        assert a in src, "mutant no longer applies: " + what
    with tempfile.TemporaryDirectory(prefix="spd_mut_") as d:
        jobs = [("control", _compile(src, d, "control"))]
        for t, (what, a, b) in enumerate(MUTANTS):
            jobs.append((what, _compile(src.replace(a, b, 1), d, "m%02d" % t)))
        with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            results = list(ex.map(lambda j: (j[0],) + _pins_pass(j[1]), jobs))
    control = results[0]
    assert control[1], "the unmutated copy must pass every pin:\n" + control[2]
    survivors = [what for what, passed, _ in results[1:] if passed]
    assert not survivors, "mutants not caught by any pin: %s" % survivors
