"""The oracle's pins catch plausible mistakes: each case plants one slip in
a copy of oracle/esmf_oracle.c (the first occurrence of the pattern;
compiled into a temporary directory) and runs the pins of
tests/test_oracle_pins.py (s functions), tests/test_angular_pins.py (the
Obara-Saika path of p and d functions) or tests/test_screening_pins.py (the
pair and density rules) against it in a child process, which
must report failing tests; likewise slips planted in a copy of
oracle/esmf_energy.py, loaded in place of the module, against
tests/test_energy_pins.py.  The unmodified copies, built and loaded the same
way, pass.  CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "esmf_oracle.c")

MUTANTS = {
    "boys_series_term": ("T * T / 10.0", "T * T / 5.0"),
    "boys_erf_argument": ("* erf(sqrt(T));", "* erf(T);"),
    "eri_prefactor": ("return 2.0 * pow(OR_PI, 2.5) / (p * q * sqrt(p + q)) *",
                      "return 2.0 * pow(OR_PI, 2.0) / (p * q * sqrt(p + q)) *"),
    "eri_exponent_sign": ("exp(-a * b / p * ab2) * exp(-c * d / q * cd2) * oracle_boys0(T);",
                          "exp(-a * b / p * ab2) * exp(c * d / q * cd2) * oracle_boys0(T);"),
    "product_center_weights": ("P[x] = (a * A[x] + b * B[x]) / p;", "P[x] = (b * A[x] + a * B[x]) / p;"),
    "primitive_norm_power": ("w[k] = c * coefs[k] * pow(2.0 * exps[k] / OR_PI, 0.75);",
                             "w[k] = c * coefs[k] * pow(2.0 * exps[k] / OR_PI, 0.5);"),
    "contracted_overlap_power": ("double ov = pow(2.0 * sqrt(ak * al) / (ak + al), 1.5);",
                                 "double ov = pow(2.0 * sqrt(ak * al) / (ak + al), 0.5);"),
    "orbit_not_deduplicated": ("if (dup) continue;", "if (0 && dup) continue;"),
    "unique_exchange_operand": ("K[k * nn + (int64_t)i0 * n + i2] += Dk[(int64_t)i1 * n + i3] * v;",
                                "K[k * nn + (int64_t)i0 * n + i2] += Dk[(int64_t)i3 * n + i1] * v;"),
    "schwarz_without_root": ("Q[(int64_t)p * n + q] = sqrt(v > 0.0 ? v : 0.0);",
                             "Q[(int64_t)p * n + q] = (v > 0.0 ? v : 0.0);"),
    "brute_exchange_operand": ("K[k * nn + (int64_t)p * n + r] += Dk[(int64_t)q * n + s] * v;",
                               "K[k * nn + (int64_t)p * n + r] += Dk[(int64_t)s * n + q] * v;"),
}


# planted in the Obara-Saika path (p and d functions), caught by tests/test_angular_pins.py
ANGULAR_MUTANTS = {
    "vrr_bra_rho_sign": ("- o->rho / o->p * os_vrr(o, e2, f, m + 1)", "+ o->rho / o->p * os_vrr(o, e2, f, m + 1)"),
    "vrr_cross_exponent": ("v += f[i] / (2.0 * (o->p + o->q)) * os_vrr(o, e1, f1, m + 1);",
                           "v += f[i] / (2.0 * o->p) * os_vrr(o, e1, f1, m + 1);"),
    "vrr_ket_boys_order": ("o->WQ[i] * os_vrr(o, e, f1, m + 1)", "o->WQ[i] * os_vrr(o, e, f1, m)"),
    "hrr_bra_sign": ("+ AB[j] * os_hrr(o, AB, CD, a, b1, c, d)", "- AB[j] * os_hrr(o, AB, CD, a, b1, c, d)"),
    "hrr_ket_sign": ("+ CD[j] * os_hrr(o, AB, CD, a, b, c, d1)", "- CD[j] * os_hrr(o, AB, CD, a, b, c, d1)"),
    "d_double_factorial": ("return l == 2 ? 3.0 : 1.0;", "return l == 2 ? 2.0 : 1.0;"),
    "d_label_table": ("{1, 1, 0}, {1, 0, 1}, {0, 1, 1}", "{1, 0, 1}, {1, 1, 0}, {0, 1, 1}"),
    "gaussian_product_point_w": ("W[x] = (p * P[x] + q * Q[x]) / (p + q);", "W[x] = (q * P[x] + p * Q[x]) / (p + q);"),
}


# planted in the screening rules, caught by tests/test_screening_pins.py
SCREENING_MUTANTS = {
    "pair_max_one_pair_only": ("if (v > *a2) *a2 = v;", ";"),
    "pair_max_skips_diagonal": ("if (r == p && s > q) continue;", "if (r == p && s >= q) continue;"),
    "density_weight_untransposed": ("double b = fabs(D[k * nn + (int64_t)y * n + x]);",
                                    "double b = fabs(D[k * nn + (int64_t)x * n + y]);"),
    "density_weight_missing_pair": ("Wd[(int64_t)p * n + r]};", "Wd[(int64_t)r * n + s]};"),
    "density_rule_factor": ("* wt < tol_d) continue;", "* wt * 0.25 < tol_d) continue;"),
}


def run_pins(tmp_path, name, pat=None, new=None, pins="test_oracle_pins.py"):
    src = open(SRC).read()
    if pat is not None:
        assert pat in src, f"pattern of {name} not in the oracle"
        src = src.replace(pat, new, 1)
    c = tmp_path / f"{name}.c"
    c.write_text(src)
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-fno-fast-math", "-ffp-contract=off",
                    str(c), "-o", str(so), "-lm"], check=True)
    env = dict(os.environ, ESMF_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins),
                        "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.mark.parametrize("pins", ["test_oracle_pins.py", "test_angular_pins.py", "test_screening_pins.py"])
def test_unmodified_copy_passes(tmp_path, pins):
    rc, out = run_pins(tmp_path, "unmodified", pins=pins)
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_slip_fails_a_pin(tmp_path, name):
    rc, out = run_pins(tmp_path, name, *MUTANTS[name])
    assert rc == 1 and "failed" in out, out


@pytest.mark.parametrize("name", sorted(ANGULAR_MUTANTS))
def test_planted_angular_slip_fails_a_pin(tmp_path, name):
    rc, out = run_pins(tmp_path, name, *ANGULAR_MUTANTS[name], pins="test_angular_pins.py")
    assert rc == 1 and "failed" in out, out


@pytest.mark.parametrize("name", sorted(SCREENING_MUTANTS))
def test_planted_screening_slip_fails_a_pin(tmp_path, name):
    rc, out = run_pins(tmp_path, name, *SCREENING_MUTANTS[name], pins="test_screening_pins.py")
    assert rc == 1 and "failed" in out, out


# planted in the energy / GVP oracle (oracle/esmf_energy.py), caught by tests/test_energy_pins.py
ENERGY_MUTANTS = {
    "norm_N2": ("N2 = c0 * c0 + 2.0 * float(np.sum(sigma * sigma))", "N2 = c0 * c0 + float(np.sum(sigma * sigma))"),
    "e1_cross_coefficient": ("+ 4.0 * c0 * np.trace(Th @ G @ Ga.T @ sigma.T)",
                             "+ 2.0 * c0 * np.trace(Th @ G @ Ga.T @ sigma.T)"),
    "density_A_sign": ("A = Ga.T @ sigma.T @ sigma @ Ga - Th.T @ sigma @ sigma.T @ Th",
                       "A = Ga.T @ sigma.T @ sigma @ Ga + Th.T @ sigma @ sigma.T @ Th"),
    "fock_exchange_sign": ("return 2.0 * J - K", "return 2.0 * J + K"),
    "dc0_normalisation_term": ("+ 2.0 * c0 * dot(FP, P) + 4.0 * dot(FP, T)) / N2 - 2.0 * c0 * E / N2",
                               "+ 2.0 * c0 * dot(FP, P) + 4.0 * dot(FP, T)) / N2"),
    "dsigma_exchange_sign": ("- 4.0 * (Th @ FP @ Th.T @ s)", "+ 4.0 * (Th @ FP @ Th.T @ s)"),
    "dtheta_transpose": ("+ 4.0 * c0 * (Th @ (FT + FT.T))", "+ 4.0 * c0 * (Th @ (FT + FT))"),
    "dgamma_transpose": ("+ 4.0 * (s.T @ Th @ FT)) / N2", "+ 4.0 * (s.T @ Th @ FT.T)) / N2"),
    "gvp_rotation_norm": ("+ 0.5 * float(np.sum(Gx * Gx))", "+ 1.0 * float(np.sum(Gx * Gx))"),
    "gvp_variance_sign": ("chi * (-2.0 * mu * (omega - E))", "chi * (2.0 * mu * (omega - E))"),
    "gvp_tangent_half": ("- 0.5 * (Adir @ Gam + Gam @ Adir)", "- 1.0 * (Adir @ Gam + Gam @ Adir)"),
}

ENERGY_RUNNER = """
import importlib.util, sys
import pytest
sys.path.insert(0, sys.argv[1])
import oracle
spec = importlib.util.spec_from_file_location("oracle.esmf_energy", sys.argv[2])
mod = importlib.util.module_from_spec(spec)
sys.modules["oracle.esmf_energy"] = mod
spec.loader.exec_module(mod)
oracle.esmf_energy = mod
sys.exit(pytest.main([sys.argv[3], "-x", "-q", "-p", "no:cacheprovider"]))
"""


def run_energy_pins(tmp_path, name, pat=None, new=None):
    src = open(os.path.join(ROOT, "oracle", "esmf_energy.py")).read()
    if pat is not None:
        assert src.count(pat) == 1, f"pattern of {name} not once in the energy oracle"
        src = src.replace(pat, new)
    f = tmp_path / f"{name}.py"
    f.write_text(src)
    r = subprocess.run([sys.executable, "-c", ENERGY_RUNNER, ROOT, str(f),
                        os.path.join(ROOT, "tests", "test_energy_pins.py")],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


def test_unmodified_energy_copy_passes(tmp_path):
    rc, out = run_energy_pins(tmp_path, "unmodified")
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(ENERGY_MUTANTS))
def test_planted_energy_slip_fails_a_pin(tmp_path, name):
    rc, out = run_energy_pins(tmp_path, name, *ENERGY_MUTANTS[name])
    assert rc == 1 and "failed" in out, out
