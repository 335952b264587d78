"""Planted mistakes: each mutation of a copy of oracle.c (a flipped sign, a
dropped term, an off-by-one, a reversed loop) must make the pin suite fail.
The mutated copy is built in a temporary directory; the real oracle is never
touched."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTATIONS = {
    "tau_sign": ("tau[j] = (beta - alpha) / beta;", "tau[j] = (alpha - beta) / beta;"),
    "beta_sign": ("double beta = (alpha >= 0.0) ? -norm : norm;",
                  "double beta = (alpha >= 0.0) ? norm : -norm;"),
    "dropped_diag_term": ("double s = A_(j, k);", "double s = 0.0;"),
    "rotation_sign": ("A_(k, i) = c * ai - s * aj;", "A_(k, i) = c * ai + s * aj;"),
    "mean_off_by_one": ("xbar = s / (double)M;", "xbar = s / (double)(M + 1);"),
    "weight_not_sqrt": ("double sw = w ? sqrt(w[n]) : 1.0;", "double sw = w ? w[n] : 1.0;"),
    "applyq_order": ("for (int64_t j = m - 1; j >= 0; --j) {\n    if (tau[j] == 0.0) continue;",
                     "for (int64_t j = 0; j < m; ++j) {\n    if (tau[j] == 0.0) continue;"),
    "truncation_strict": ("if (acc / total >= energy)", "if (acc / total > energy)"),
    "transposed_vt": ("VT[k * ldvt + i] = V[i * M + k];", "VT[k * ldvt + i] = V[k * M + i];"),
    "grad_factor": ("double g = 2.0 * (Y[m * N + n] - p) * swn;", "double g = 1.0 * (Y[m * N + n] - p) * swn;"),
    "zqr_missing_conj": ("for (int64_t i = j + 1; i < n; ++i) s += conj(Z_(i, j)) * Z_(i, k);",
                         "for (int64_t i = j + 1; i < n; ++i) s += Z_(i, j) * Z_(i, k);"),
    "zjacobi_phase": ("zc eph = conj(gamma) / g; /* e^{-i phi} */", "zc eph = gamma / g; /* e^{-i phi} */"),
    "zsvd_phase_rule": ("zc ph = (vmax > 0.0) ? conj(Vw[p * M + kmax]) / vmax : 1.0;",
                        "zc ph = (vmax > 0.0) ? Vw[p * M + kmax] / vmax : 1.0;"),
    "grad_weight_missing": ("double g = 2.0 * (Y[m * N + n] - p) * swn;", "double g = 2.0 * (Y[m * N + n] - p);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    # the first occurrence is mutated (the real routines precede the complex ones)
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = tmp_path / "oracle_mut.c"
    mutated.write_text(src.replace(old, new, 1))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", str(lib),
                    str(mutated), "-lm"], check=True)
    env = dict(os.environ, PYLOM_ORACLE_LIB=str(lib), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutation {name}:\n{r.stdout[-2000:]}"
