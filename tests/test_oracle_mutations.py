"""Planted mistakes in the oracle: the pins must catch each one (CPU only).

Each case below is a plausible slip in one step of the FP64 oracle: a dropped
factor or term, a wrong sign, index or direction, a transposed operand.  The
test copies the oracle (C source and Python modules), the oracle's pin files
and the pure-Python workload module into a scratch directory, plants one
mistake in the copy, and runs the pins there in a subprocess: at least one pin
must fail.  An unmutated copy must pass them all, so a failure is the planted
mistake's and not the harness's.  The committed oracle is never touched.

Steps covered (Kitzmann et al. 2020): Gauss-Legendre angles and the flux
quadrature (Eq. 8), short characteristics with a linear source (Eqs. 4-7) and
the parabolic moments, the Planck function (Eq. 2), the bilinear log10 sigma
and log10 CIA interpolation and the abundance-weighted sum (Sects. 2.3, 2.8),
the mean molecular weight and H2/He split, the hydrostatic trapezoid optical
depth, the finite-element temperature profile (Sect. 2.5.1, Eqs. 12-16) and
Milne's profile (Sect. 2.5), the distance scaling (Eq. 9), the instrument
profile (Eq. 17) and binning, the likelihood and its error inflation
(Eqs. 22-23), the gray cloud, the Hopf function and the nested-sampling shell
weights.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PIN_FILES = ["test_oracle_pins.py", "test_oracle_parabolic.py", "test_oracle_cloud.py",
             "test_oracle_milne.py", "test_nested_oracle.py"]

C = "hr2_oracle.c"
# (id, file under oracle/, text in the committed source (exactly once), replacement)
MUTATIONS = [
    ("gl_weight_half_dropped", C, "w[n - 1 - i] = 0.5 * wx;", "w[n - 1 - i] = wx;"),
    ("flux_mu_weight_dropped", C, "F += w[k] * mu[k] * or_sc_intensity(L,", "F += w[k] * or_sc_intensity(L,"),
    ("sc_beta_gamma_swapped", C, "I = I * e + beta * S[l] + gamma * S[l + 1];",
     "I = I * e + gamma * S[l] + beta * S[l + 1];"),
    ("sc_gamma_transmission_dropped", C, "double gamma = q - e;", "double gamma = q;"),
    ("parabolic_m2_factor", C, "*M2 = 2.0 * *M1 - D * D * e;", "*M2 = *M1 - D * D * e;"),
    ("parabolic_series_index", C, "s[k] += term * pow(D, k) / (double)(k + n + 1);",
     "s[k] += term * pow(D, k) / (double)(n + 1);"),
    ("planck_nu_squared", C, "return 2.0 * OR_H * OR_C * OR_C * nu * nu * nu / expm1(x);",
     "return 2.0 * OR_H * OR_C * OR_C * nu * nu / expm1(x);"),
    ("planck_wien", C, "nu * nu * nu / expm1(x);", "nu * nu * nu / exp(x);"),
    ("sigma_corners_inconsistent", C,
     "double v = (1.0 - wT) * (1.0 - wp) * OR_TAB(a, b) + wT * (1.0 - wp) * OR_TAB(a + 1, b) +",
     "double v = (1.0 - wT) * (1.0 - wp) * OR_TAB(a, b) + wp * (1.0 - wT) * OR_TAB(a + 1, b) +"),
    ("cia_weights_swapped", C,
     "return (1.0 - wT) * cia[(size_t)a * m->n_nu_tab + inu] + wT * cia[(size_t)(a + 1) * m->n_nu_tab + inu];",
     "return wT * cia[(size_t)a * m->n_nu_tab + inu] + (1.0 - wT) * cia[(size_t)(a + 1) * m->n_nu_tab + inu];"),
    ("abundance_of_first_absorber_for_all", C, "chi += st->x[s] * or_sigma(m, m->species[s],",
     "chi += st->x[0] * or_sigma(m, m->species[s],"),
    ("sigma_by_setup_index", C, "chi += st->x[s] * or_sigma(m, m->species[s],", "chi += st->x[s] * or_sigma(m, s,"),
    ("last_absorber_dropped", C, "for (int s = 0; s < m->n_used; ++s)\n    chi += st->x[s]",
     "for (int s = 0; s + 1 < m->n_used; ++s)\n    chi += st->x[s]"),
    ("mass_by_setup_index", C, "mmw += st->x[s] * m->species_mass[m->species[s]];",
     "mmw += st->x[s] * m->species_mass[s];"),
    ("helium_ratio_dropped", C, "st->x_he = m->r_he * st->x_h2;", "st->x_he = st->x_h2;"),
    ("dtau_trapezoid_half_dropped", C, "    dtau[l] = 0.5 * (chi[l] + chi[l + 1]) * (st->p[l + 1] - st->p[l]) * colfac",
     "    dtau[l] = (chi[l] + chi[l + 1]) * (st->p[l + 1] - st->p[l]) * colfac"),
    ("top_flux_bottom_boundary", C, "return or_sc_flux(L, dtau, S, S[L], m->n_mu);",
     "return or_sc_flux(L, dtau, S, S[L - 1], m->n_mu);"),
    ("top_flux_cloud_dropped", C,
     "(st->p[l + 1] - st->p[l]) * colfac + st->tau_cloud[l];\n  if (m->sc_order == 2)",
     "(st->p[l + 1] - st->p[l]) * colfac;\n  if (m->sc_order == 2)"),
    ("fe_profile_upside_down", C, "(double)(L - j) / (double)L", "(double)j / (double)L"),
    ("fe_global_dof_index", C, "T += Tnodes[k * q + i]", "T += Tnodes[k + i]"),
    ("fe_ratios_from_bottom_node", C, "Tnodes[i] = b[i - 1] * Tnodes[i - 1];", "Tnodes[i] = b[i - 1] * Tnodes[0];"),
    ("milne_three_quarters_dropped", C, "return pow(0.75 * pow(Tbar, 4.0) * (tau + or_hopf(m, tau)), 0.25);",
     "return pow(pow(Tbar, 4.0) * (tau + or_hopf(m, tau)), 0.25);"),
    ("distance_scaling_not_squared", C, "st->scale = f * (m->radius_cm / d) * (m->radius_cm / d);",
     "st->scale = f * (m->radius_cm / d);"),
    ("bin_mean_count", C, "else bins[b] = sum / cnt;", "else bins[b] = sum / (cnt + 1);"),
    ("lnl_two_pi_dropped", C, "lnL += -r * r / (2.0 * s2) - 0.5 * log(2.0 * M_PI * s2);",
     "lnL += -r * r / (2.0 * s2) - 0.5 * log(M_PI * s2);"),
    ("error_inflation_not_exponentiated", C, "if (isfinite(log_eps)) s2 += pow(10.0, log_eps);",
     "if (isfinite(log_eps)) s2 += log_eps;"),
    ("cloud_spread_over_wrong_range", C, "if (hi > lo) st->tau_cloud[l] = tc * (hi - lo) / (pb - pt);",
     "if (hi > lo) st->tau_cloud[l] = tc * (hi - lo) / pb;"),
    ("hopf_source_half_dropped", "hopf.py", "0.5 * _en(3, t)", "_en(3, t)"),
    ("nested_shell_index", "nested.py", "return -(i - 1) / n_live + math.log(-math.expm1(-1.0 / n_live))",
     "return -i / n_live + math.log(-math.expm1(-1.0 / n_live))"),
]


def _scratch(tmp_path, mutation=None):
    """The scratch tree: oracle/ (one mistake planted), tests/ (the pin files
    and the suite's conftest), paper_1910_01070_b300/ (the workload module
    only), pytest.ini."""
    d = tmp_path / "tree"
    (d / "oracle").mkdir(parents=True)
    (d / "tests").mkdir()
    (d / "paper_1910_01070_b300").mkdir()
    for f in ("__init__.py", "hopf.py", "nested.py", C):
        shutil.copy(os.path.join(ROOT, "oracle", f), d / "oracle" / f)
    for f in ["conftest.py"] + PIN_FILES:
        shutil.copy(os.path.join(ROOT, "tests", f), d / "tests" / f)
    for f in ("__init__.py", "workloads.py"):
        shutil.copy(os.path.join(ROOT, "paper_1910_01070_b300", f), d / "paper_1910_01070_b300" / f)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d / "pytest.ini")
    if mutation is not None:
        _, fname, old, new = mutation
        path = d / "oracle" / fname
        src = path.read_text()
        assert src.count(old) == 1, "mutation target not found exactly once: %r" % old
        path.write_text(src.replace(old, new))
    return d


def _run_pins(d):
    env = dict(os.environ)
    env.pop("PYTHONPATH", None)
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu"] +
                          ["tests/" + f for f in PIN_FILES],
                          cwd=str(d), env=env, capture_output=True, text=True, timeout=600)


def test_unmutated_copy_passes_the_pins(tmp_path):
    r = _run_pins(_scratch(tmp_path))
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "passed" in r.stdout and "failed" not in r.stdout


@pytest.mark.parametrize("mutation", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, mutation):
    r = _run_pins(_scratch(tmp_path, mutation))
    # exit code 1: tests ran and at least one failed (not a collection or
    # build error, which would say nothing about the pins)
    assert r.returncode == 1, (mutation[0], r.returncode, r.stdout[-1500:], r.stderr[-1500:])
    assert "1 failed" in r.stdout, r.stdout[-1500:]
