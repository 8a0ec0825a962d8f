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


# ---- the subgrid producer's oracle (oracle/predict.py) ----------------------

PREDICT_SRC = os.path.join(ROOT, "oracle", "predict.py")

PREDICT_MUTANTS = {
    "w_phase_sign": ("np.exp(-2j * np.pi * (turns_uv + w * nm1))", "np.exp(-2j * np.pi * (turns_uv - w * nm1))"),
    "l_m_swapped": ("turns_uv = ((u0 * a[None, :] + v0 * a[:, None]) % N)",
                    "turns_uv = ((u0 * a[:, None] + v0 * a[None, :]) % N)"),
    "shift_order": ("np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(J)))", "np.fft.fftshift(np.fft.fft2(J))"),
    "inverse_transform": ("np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(J)))",
                          "np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(J))) * N * N"),
    "plane_spacing": ("J = img * T * _screen(N, theta, int(u0), int(v0), w0 + c * dw)",
                      "J = img * T * _screen(N, theta, int(u0), int(v0), w0 + c * dw * 0.5)"),
    "taper_dropped": ("J = img * T * _screen(", "J = img * _screen("),
    "pixel_centre_off_by_one": ("idx = (np.arange(N, dtype=np.float64) - N // 2) * (theta / N)",
                                "idx = (np.arange(N, dtype=np.float64) - N // 2 + 1) * (theta / N)"),
}


@pytest.mark.parametrize("name", ["unchanged"] + sorted(PREDICT_MUTANTS))
def test_predict_pins_kill_mutant(name, tmp_path):
    # "unchanged" runs the harness on the oracle as it is: the pins pass
    before, after = PREDICT_MUTANTS.get(name, ("", ""))
    src = open(PREDICT_SRC).read()
    assert before in src, "mutation site not found: update the mutant"
    pkg = tmp_path / "mutpkg" / "oracle"
    pkg.mkdir(parents=True)
    (pkg / "__init__.py").write_text("")
    (pkg / "predict.py").write_text(src.replace(before, after, 1))
    # the pins run from a copy beside the mutated package, so that `oracle`
    # resolves to the mutant and not to the repository's package
    test = tmp_path / "mutpkg" / "test_pins.py"
    test.write_text(open(os.path.join(ROOT, "tests", "test_oracle_predict.py")).read())
    env = dict(os.environ, PYTHONPATH=str(tmp_path / "mutpkg"))
    probe = subprocess.run([sys.executable, "-c", "import oracle.predict as m; print(m.__file__)"],
                           cwd=str(tmp_path / "mutpkg"), env=env, capture_output=True, text=True)
    assert probe.stdout.strip() == str(pkg / "predict.py"), probe.stdout + probe.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "--rootdir",
                        str(tmp_path / "mutpkg"), "-c", os.devnull, str(test)],
                       cwd=str(tmp_path / "mutpkg"), env=env, capture_output=True, text=True, timeout=600)
    assert "ModuleNotFoundError" not in r.stdout + r.stderr, r.stdout[-2000:]
    if name == "unchanged":
        assert r.returncode == 0, r.stdout[-2000:]
    else:
        assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
