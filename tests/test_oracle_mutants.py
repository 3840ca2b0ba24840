"""The pins have teeth: each planted mistake in a copy of the oracle's C
source makes at least one pin of tests/test_oracle_pins.py fail.

Every mutant is a plausible slip in one equation of the method -- a prior
gradient, the dispersion, the Langevin noise scale, a transposed index, the
part rule of Sec. 3, the stochastic-gradient scale N / |Pi_t|, the step-size
schedule, the Tweedie power and its clamp below mu_min (in the gradient and
in the log-likelihood), the mirror, the uniform and Box-Muller steps of the
noise, the beta divergence and the posterior variance.  The mutant is
compiled into a library of its own in a temporary directory and the pin
suite runs against it in a child process (the oracle's loader reads the
source and library paths from PSGLD_ORACLE_SOURCE / PSGLD_ORACLE_LIB); the
committed oracle is never touched.  CPU only.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "psgld_oracle.c")
HDR = os.path.join(ROOT, "oracle", "psgld_oracle.h")

# name: (exact text in the oracle, the mistake)
MUTANTS = {
    "gaussian_prior_without_square": (
        "return -x / (s * s);", "return -x / s;"),
    "exponential_prior_sign": (
        "return mat == 0 ? -m->lambda_w : -m->lambda_h;",
        "return mat == 0 ? m->lambda_w : -m->lambda_h;"),
    "dispersion_dropped": (
        "return (v - mu) * pow(mc, -m->p) / m->phi;", "return (v - mu) * pow(mc, -m->p);"),
    "tweedie_power_sign": (
        "return (v - mu) * pow(mc, -m->p) / m->phi;", "return (v - mu) * pow(mc, m->p) / m->phi;"),
    "noise_scale_sqrt_eps": (
        "const double sd = sqrt(2.0 * eps);", "const double sd = sqrt(eps);"),
    "transposed_H_index_in_mu": (
        "mu += m->W[i * K + k] * m->H[(int64_t)k * J + j];",
        "mu += m->W[i * K + k] * m->H[(int64_t)j * K + k];"),
    "part_rule_shifted": (
        "return (int32_t)((r + s) % B);", "return (int32_t)((r + s + 1) % B);"),
    "scale_B_instead_of_N_over_part": (
        "return n > 0 ? (double)m->N / (double)n : 0.0;", "return (double)m->B;"),
    "step_size_off_by_one": (
        "return pow(m->eps_a / (double)t, m->eps_b);",
        "return pow(m->eps_a / (double)(t + 1), m->eps_b);"),
    "mirror_dropped_on_W": (
        "m->W[a] = mirror ? fabs(w) : w;", "m->W[a] = w;"),
    "uniform_scale": (
        "u[n] = ((double)(x[n] >> 9) + 0.5) / 8388608.0;",
        "u[n] = ((double)(x[n] >> 9) + 0.5) / 8388609.0;"),
    "box_muller_swapped_radius": (
        "z[1] = r0 * sin(two_pi * u[1]);", "z[1] = r1 * sin(two_pi * u[1]);"),
    "beta_divergence_general_term": (
        "- v * pow(mu, beta - 1.0) / (beta - 1.0)", "- v * pow(mu, beta - 1.0) / beta"),
    "mu_min_clamps_the_residual_too": (
        "return (v - mu) * pow(mc, -m->p) / m->phi;", "return (v - mc) * pow(mc, -m->p) / m->phi;"),
    "mu_min_clamp_dropped_in_gradient": (
        "double mc = mu > m->mu_min ? mu : m->mu_min;", "double mc = mu;"),
    "mu_min_clamp_dropped_in_log_lik": (
        "if (m->p > 0.0 && mu < m->mu_min) mu = m->mu_min;", "if (0) mu = m->mu_min;"),
    "posterior_variance_without_square": (
        "Wvar[a] = n > 0 ? m->sW2[a] / n - mean * mean : 0.0;",
        "Wvar[a] = n > 0 ? m->sW2[a] / n - mean : 0.0;"),
}


def _run_pins(name, tmp):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, (name, "the text to mutate must occur exactly once")
    d = os.path.join(tmp, name)
    os.makedirs(d)
    with open(os.path.join(d, "psgld_oracle.c"), "w") as f:
        f.write(src.replace(old, new))
    shutil.copy(HDR, d)
    lib = os.path.join(d, "liboracle_psgld.so")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", "-o", lib, os.path.join(d, "psgld_oracle.c"), "-lm"])
    env = dict(os.environ, PSGLD_ORACLE_SOURCE=os.path.join(d, "psgld_oracle.c"),
               PSGLD_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                        "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    failed = [ln.split("::", 1)[1].split(" ")[0] for ln in r.stdout.splitlines()
              if ln.startswith("FAILED ")]
    return r.returncode, failed, r.stdout[-2000:]


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    tmp = str(tmp_path_factory.mktemp("mutants"))
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        futs = {n: ex.submit(_run_pins, n, tmp) for n in MUTANTS}
        return {n: f.result() for n, f in futs.items()}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(results, name):
    rc, failed, tail = results[name]
    # 1 = some test failed (not a crash, a collection error or a timeout)
    assert rc == 1 and failed, (name, rc, tail)
