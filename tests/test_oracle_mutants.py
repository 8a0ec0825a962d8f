"""The oracle's pins must fail on plausible mistakes (CPU only).

Each case plants one mistake in a temporary copy of ``oracle/oracle.c``
(never the file itself), compiles it, and runs the pin tests of
``test_oracle.py`` against that copy in a subprocess; the run must fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "start_off_by_one": ("long long s = i - W / 2 + 1;", "long long s = i - W / 2;"),
    "floor_instead_of_rint": ("long long p = llrint(qo);", "long long p = (long long)floor(qo);"),
    "v_row_from_u": ("const double *gv = g_uv + c.fv * uv_support;\n                const double *gw",
                     "const double *gv = g_uv + c.fu * uv_support;\n                const double *gw"),
    "dropped_w_term": ("for (int k = 0; k < w_support; ++k) {\n                            double w = gv[b] * gu[a] * gw[k];\n                            int64_t e = ((c.y0 + b) * nx + (c.x0 + a)) * nz + (c.z0 + k);\n                            re",
                       "for (int k = 1; k < w_support; ++k) {\n                            double w = gv[b] * gu[a] * gw[k];\n                            int64_t e = ((c.y0 + b) * nx + (c.x0 + a)) * nz + (c.z0 + k);\n                            re"),
    "x_y_transposed": ("int64_t e = ((c.y0 + b) * nx + (c.x0 + a)) * nz + (c.z0 + k);\n                            re +=",
                       "int64_t e = ((c.x0 + a) * nx + (c.y0 + b)) * nz + (c.z0 + k);\n                            re +="),
    "imag_sign": ("im += w * sg[2 * e + 1];", "im -= w * sg[2 * e + 1];"),
    "reversed_table_row": ("double w = gv[b] * gu[a] * gw[k];\n                            int64_t e = ((c.y0 + b) * nx + (c.x0 + a)) * nz + (c.z0 + k);\n                            re",
                           "double w = gv[uv_support - 1 - b] * gu[a] * gw[k];\n                            int64_t e = ((c.y0 + b) * nx + (c.x0 + a)) * nz + (c.z0 + k);\n                            re"),
    "adjoint_mixes_re_im": ("sg[2 * e] += w * yre;", "sg[2 * e] += w * yim;"),
    "bounds_off_by_one": ("return s >= 0 && s <= (long long)n - W;", "return s >= 0 && s <= (long long)n - W + 1;"),
    "2d_offsets_swapped": ("((int64_t)c.fv * uv_oversample + c.fu) * block;", "((int64_t)c.fu * uv_oversample + c.fv) * block;"),
    "2d_block_transposed": ("double w = G[b * uv_support + a] * gw[k];", "double w = G[a * uv_support + b] * gw[k];"),
    "2d_adjoint_block_transposed": ("double w = G[b * uv_support + a] * gw[k];\n                        int64_t e = ((c.y0 + b) * nx + (c.x0 + a)) * nz + (c.z0 + k);\n                        sg[2 * e] += w * yre;",
                                    "double w = G[a * uv_support + b] * gw[k];\n                        int64_t e = ((c.y0 + b) * nx + (c.x0 + a)) * nz + (c.z0 + k);\n                        sg[2 * e] += w * yre;"),
    "2d_x_y_transposed": ("double w = G[b * uv_support + a] * gw[k];\n                            int64_t e = ((c.y0 + b) * nx + (c.x0 + a)) * nz + (c.z0 + k);",
                          "double w = G[b * uv_support + a] * gw[k];\n                            int64_t e = ((c.x0 + a) * nx + (c.y0 + b)) * nz + (c.z0 + k);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_kill_mutant(name, tmp_path):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert before in src, "mutation site not found: update the mutant"
    mutated = tmp_path / "oracle_mutant.c"
    mutated.write_text(src.replace(before, after, 1))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                    "-shared", str(mutated), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB=str(lib), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
