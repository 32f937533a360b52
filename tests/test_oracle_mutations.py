"""Planted mistakes in the oracle must be caught by its pins.

Each case copies oracle/fdlb_oracle.c, plants one plausible mistake (a dropped
term, a wrong coefficient, sign or index), builds it into a temporary library
and runs tests/test_oracle_pins.py against it in a subprocess; the pins must
fail.  Everything runs on the CPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fdlb_oracle.c")

MUTATIONS = {
    "j1_theta_dlnT_coeff": ("0.3 * (xi * xi * xi / T + 7.0 * xi / 3.0) * dlnT", "0.3 * (xi * xi * xi / T + xi / 3.0) * dlnT"),
    "j1_phi_missing_Y": ("j1phi[k] = -Y * bphi * fmb[k];", "j1phi[k] = -bphi * fmb[k];"),
    "j1_phi_du_coeff": ("0.6 * (xi * xi / T - 1.0) * du +", "0.6 * (xi * xi / T - 1.0 / 3.0) * du +"),
    "shakhov_phi_poly": ("(1.0 + a * (xi * xi / T - 3.0) * xi * q)", "(1.0 + a * (xi * xi / T - 1.0) * xi * q)"),
    "weno_weight_power": ("s += d[r] * (t * t);", "s += d[r] * t;"),
    "weno_candidate_sign": ("F3 = f0 / 3.0 + 5.0 * fp1 / 6.0 - fp2 / 6.0", "F3 = f0 / 3.0 + 5.0 * fp1 / 6.0 + fp2 / 6.0"),
    "weno_mirror_index": ("s[r] = ef[(size_t)(j + 3 - r) * Q + k];", "s[r] = ef[(size_t)(j + 2 - r) * Q + k];"),
    "cd6_coeff": ("3.0 * q[4] / 4.0", "3.0 * q[4] / 5.0"),
    "rk3_stage2": ("p2[e] = 0.75 * phi[e] + 0.25 * p1[e] + 0.25 * dt * Lp[e];", "p2[e] = 0.75 * phi[e] + 0.25 * p1[e] + 0.5 * dt * Lp[e];"),
    "moments_temperature": ("out[2] = e / (1.5 * n);", "out[2] = e / n;"),
    "equilibrium_order": ("int N = Q - 1;", "int N = Q - 2;"),
    "chi_sign": ("return 0.5 * (2.0 - eta) / pow(1.0 - eta, 3.0);", "return 0.5 * (2.0 + eta) / pow(1.0 - eta, 3.0);"),
    "viscosity_coeff": ("(1.0 / Y + 0.8 + 4.0 / 25.0", "(1.0 / Y + 1.2 + 4.0 / 25.0"),
    "dlnchi_chain_rule": ("eta * (3.0 / (1.0 - eta) - 1.0 / (2.0 - eta)) * dlnrho", "eta * (2.0 / (1.0 - eta) - 1.0 / (2.0 - eta)) * dlnrho"),
    "ghost_theta": ("for (int k = 0; k < Q; ++k) dt[k] = 2.0 * s[2] * dp[k];", "for (int k = 0; k < Q; ++k) dt[k] = s[2] * dp[k];"),
    "rh_energy": ("double e1 = 1.5 * rho1 * T1", "double e1 = 2.5 * rho1 * T1"),
    "prandtl_coeff": ("double den = 1.0 + 1.2 * Y", "double den = 1.0 + 1.0 * Y"),
    "sound_init_eos": ("T[c] = P0 / (r * (1.0 + 4.0 * eta * oq_chi_set(eta)));", "T[c] = P0 / (r * (1.0 + 2.0 * eta * oq_chi_set(eta)));"),
    "quadrature_weight": ("w[k] = qf / (hq1 * hq1);", "w[k] = qf / (hq1 * hq1) * (1.0 + 1e-9 * k);"),
    "fm_slice_area": ("double Fb = sigma * sigma * b - b * b * b / 3.0;", "double Fb = sigma * sigma * b - b * b * b / 2.0;"),
    "fm_normalisation": ("return 3.0 / (4.0 * sigma * sigma * sigma) * (Fb - Fa);", "return 1.0 / (sigma * sigma * sigma) * (Fb - Fa);"),
    "fm_halfwidth": ("while ((W + 0.5) * dx < sigma) ++W;", "while ((W + 1.0) * dx < sigma) ++W;"),
    "fm_fixed_extension": ("src = jj < 0 ? 0 : (jj >= ne ? ne - 1 : jj);", "src = jj < 0 ? 0 : (jj >= ne ? 0 : jj);"),
    "fm_periodic_wrap": ("src = ((i % nx) + nx) % nx + OQ_NG;", "src = ((i % nx) + nx) % nx;"),
    "ret_dlnchi": ("double dlnchi = m->chi_mode == 1 ? oq_cd6(lnchi + j - 3, m->dx)", "double dlnchi = m->chi_mode == 1 ? 0.5 * oq_cd6(lnchi + j - 3, m->dx)"),
    "ret_tau_local_chi": ("double tau = oq_tau_chi(m, n, chi, T);", "double tau = oq_tau(m, n, T);"),
    "sound_alpha_a_gamma": ("out[1] = k * k / (2.0 * rho) * (4.0 * mu / 3.0 + muv + (gamma - 1.0) * lambda / cP);", "out[1] = k * k / (2.0 * rho) * (4.0 * mu / 3.0 + muv + gamma * lambda / cP);"),
    "sound_alpha_t_cp": ("out[3] = lambda * k * k / (rho * cP);", "out[3] = lambda * k * k / (rho * cV);"),
    "ret_prandtl_local_chi": ("double Pr = m->pr_mode == 0 ? m->pr_const : oq_prandtl_dense(Y);", "double Pr = oq_prandtl(m, n);"),
    "shakhov_theta_poly": ("thetaS[k] = 2.0 * T * fmb[k] * (1.0 + a * (xi * xi / T - 1.0) * xi * q);", "thetaS[k] = 2.0 * T * fmb[k] * (1.0 + a * (xi * xi / T - 3.0) * xi * q);"),
    "rk3_stage3": ("phi[e] = phi[e] / 3.0 + 2.0 / 3.0 * p2[e] + 2.0 / 3.0 * dt * Lp[e];", "phi[e] = phi[e] / 3.0 + 2.0 / 3.0 * p2[e] + 1.0 / 3.0 * dt * Lp[e];"),
    "rk3_theta_stage2_operand": ("t2[e] = 0.75 * theta[e] + 0.25 * t1[e] + 0.25 * dt * Lt[e];", "t2[e] = 0.75 * theta[e] + 0.25 * t1[e] + 0.25 * dt * Lp[e];"),
    "moments_pressure_tensor": ("Pi += xi * xi * phi[k];", "Pi += xi * phi[k];"),
    "moments_heat_flux": ("q += xi * ek;", "q += xi * xi * ek;"),
    "upwind_direction": ("if (pk > 0.0)", "if (pk < 0.0)"),
    "weno_zero_indicator_case": ("if (z3 && z1) { om[0] = 0.25; om[1] = 0.0; om[2] = 0.75; return; }", "if (z3 && z1) { om[0] = 0.75; om[1] = 0.0; om[2] = 0.25; return; }"),
    "j1_theta_du_coeff": ("0.6 * (xi * xi / T - 1.0 / 3.0) * du", "0.6 * (xi * xi / T - 1.0) * du"),
    "j1_phi_dlnT_coeff": ("0.3 * (xi * xi * xi / T + xi / 3.0) * dlnT", "0.3 * (xi * xi * xi / T + xi) * dlnT"),
}


@pytest.mark.slow
def test_unmutated_oracle_copy_passes(tmp_path):
    """Control: the oracle rebuilt the same way, unmutated, passes its pins, so a failure below is the
    planted mistake's and not the build's."""
    so = tmp_path / "liboracle_copy.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), SRC, "-lm"])
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=dict(os.environ, ORACLE_LIB=str(so)), capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique/found: {name}"
    mutated = tmp_path / "fdlb_oracle.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(mutated), "-lm"])
    env = dict(os.environ, ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name} passed every pin:\n{r.stdout[-2000:]}"


RIEMANN = os.path.join(ROOT, "oracle", "riemann.py")
RIEMANN_MUTATIONS = {
    "chi_sign": ("return 0.5 * (2.0 - eta) / (1.0 - eta) ** 3", "return 0.5 * (2.0 + eta) / (1.0 - eta) ** 3"),
    "eos_coeff": ("return 1.0 + 4.0 * eta * chi_set(eta)", "return 1.0 + 3.0 * eta * chi_set(eta)"),
    "rarefaction_velocity_sign": ("return c2, -math.sqrt(c2) / r", "return c2, math.sqrt(c2) / r"),
    "hugoniot_energy_factor": ("return 1.5 * (gas.temperature(r2, Pc) - TR)", "return 2.5 * (gas.temperature(r2, Pc) - TR)"),
    "shock_speed": ("xi_s = math.sqrt((Pc - PR) / (rhoR * (1.0 - rhoR / rho2)))", "xi_s = math.sqrt((Pc - PR) / (rhoR * (1.0 + rhoR / rho2)))"),
}


def _run_riemann_pins(tmp_path, old=None, new=None):
    """Runs tests/test_riemann_oracle.py against a copy of oracle/ (riemann.py optionally mutated)."""
    import shutil
    src = open(RIEMANN).read()
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("__pycache__", "*.so"))
    if old is not None:
        (tmp_path / "oracle" / "riemann.py").write_text(src.replace(old, new))
    shutil.copytree(os.path.join(ROOT, "tests"), tmp_path / "tests", ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path)
    env = dict(os.environ, PYTHONPATH=str(tmp_path))
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           "tests/test_riemann_oracle.py"], cwd=tmp_path, env=env, capture_output=True, text=True,
                          timeout=600)


@pytest.mark.slow
def test_riemann_unmutated_copy_passes(tmp_path):
    """Control: the copied, unmutated oracle passes, so a failure below is the planted mistake's."""
    r = _run_riemann_pins(tmp_path)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(RIEMANN_MUTATIONS))
def test_riemann_planted_mistake_is_caught(name, tmp_path):
    """The same for the exact dense-gas Riemann solution: a mutated copy of oracle/riemann.py, imported in
    place of the original, fails tests/test_riemann_oracle.py."""
    old, new = RIEMANN_MUTATIONS[name]
    assert open(RIEMANN).read().count(old) == 1, f"mutation anchor not unique/found: {name}"
    r = _run_riemann_pins(tmp_path, old, new)
    assert r.returncode != 0, f"planted mistake {name} passed every pin:\n{r.stdout[-2000:]}"


CLOSURE = os.path.join(ROOT, "oracle", "closure_oracle.py")
CLOSURE_MUTATIONS = {
    "zero_padding": ("return a[np.clip(idx, 0, X - 1)]", "return np.where(((idx >= 0) & (idx < X))[:, None], a[np.clip(idx, 0, X - 1)], 0.0)"),
    "tap_offset": ("z += w[j:j + X] @ W[:, j, :].T", "z += w[TAPS - 1 - j:TAPS - 1 - j + X] @ W[:, j, :].T"),
    "relu_on_output": ("a = np.maximum(z, 0.0) if l < len(layers) - 1 else z", "a = np.maximum(z, 0.0)"),
    "loss_gradient_scale": ("dz = 2.0 * d / nel", "dz = d / nel"),
    "periodic_fold": ("da[X - 2:] += dw[0:2]", "da[:2] += dw[0:2]"),
    "replicate_fold": ("da[0] += dw[0] + dw[1]", "da[0] += dw[0]"),
    "relu_gradient_mask": ("dz = da * (zs[l - 1] > 0.0)", "dz = da"),
}


def _run_closure_pins(tmp_path, old=None, new=None):
    """Runs tests/test_closure_oracle.py against a copy of oracle/ (closure_oracle.py optionally mutated)."""
    import shutil
    src = open(CLOSURE).read()
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("__pycache__", "*.so"))
    if old is not None:
        (tmp_path / "oracle" / "closure_oracle.py").write_text(src.replace(old, new))
    shutil.copytree(os.path.join(ROOT, "tests"), tmp_path / "tests", ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path)
    env = dict(os.environ, PYTHONPATH=str(tmp_path))
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           "tests/test_closure_oracle.py"], cwd=tmp_path, env=env, capture_output=True, text=True,
                          timeout=600)


@pytest.mark.slow
def test_closure_unmutated_copy_passes(tmp_path):
    """Control for the closure network oracle's planted mistakes."""
    r = _run_closure_pins(tmp_path)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(CLOSURE_MUTATIONS))
def test_closure_planted_mistake_is_caught(name, tmp_path):
    """A mutated copy of oracle/closure_oracle.py (padding, tap order, output ReLU, loss scale, the fold of
    the window gradient at the ends, the ReLU mask) fails tests/test_closure_oracle.py."""
    old, new = CLOSURE_MUTATIONS[name]
    assert open(CLOSURE).read().count(old) == 1, f"mutation anchor not unique/found: {name}"
    r = _run_closure_pins(tmp_path, old, new)
    assert r.returncode != 0, f"planted mistake {name} passed every pin:\n{r.stdout[-2000:]}"
