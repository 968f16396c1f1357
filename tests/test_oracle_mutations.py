"""Plant plausible mistakes in copies of the oracle and check that its pins
catch every one (each mutant is built from a patched copy of rt_oracle.cpp in
a temporary directory and run against the pin named beside it)."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rt_oracle.cpp")

# name: (original text, mistake, pin expected to fail)
MUTANTS = {
    "rk4_weight": ("k + scale(2.0, k2) + scale(2.0, k3) + k4", "k + scale(2.0, k2) + k3 + k4",
                   "test_rk4_fourth_order"),
    "force_sign": ("return scale(-kCpe / (2.0 * C.f * C.f), s.grad);",
                   "return scale(kCpe / (2.0 * C.f * C.f), s.grad);", "test_slab_parabola_exact"),
    "theta_grad_sign": ("-rho / r2};", "rho / r2};", "test_interpolant_reproduces_linear_field"),
    "fu_index": ("fu = fu + sg[a] * wv[b] * ww[c] * ne_c;", "fu = fu + sg[a] * wv[b] * wu[c] * ne_c;",
                 "test_interpolant_gradient_matches_finite_differences"),
    "transfer_S_inverted": ("exp(P.ln_s[i + 1] - P.ln_s[i])", "exp(P.ln_s[i] - P.ln_s[i + 1])",
                            "test_IS_conserved_without_emission"),
    "segment_mean_T": ("T tbar = 0.5 * (P.te[i] + P.te[i + 1]);", "T tbar = P.te[i];",
                       "test_transfer_matches_formal_solution"),
    "eps_ratio": ("C.o->eta * ds;", "ds;", "test_stepwise_eps_at_slab_surface"),
    "same_k_neighbours": ("Vec3<T> k = k0;\n    rk4<T>(C, nodes, r, k);",
                          "Vec3<T> k = scale(1.001, k0);\n    rk4<T>(C, nodes, r, k);",
                          "test_stepwise_small_step_law"),
    "crossing_root": ("T a = leaving ? (-B + sqrt(disc)) / (2.0 * A) : (-B - sqrt(disc)) / (2.0 * A);",
                      "T a = leaving ? (-B - sqrt(disc)) / (2.0 * A) : (-B + sqrt(disc)) / (2.0 * A);",
                      "test_uniform_medium_straight_chords"),
    "tube_pairing": ("scale(0.5, nb_r[j] - nb_r[j + 1])", "scale(0.5, nb_r[j] - rn)",
                     "test_slab_tube_lockstep_closed_form"),
    "launch_without_n": ("k0 = scale(sqrt(n2), cvt<T>(fr.d));", "k0 = cvt<T>(fr.d);",
                         "test_bouguer_invariant_and_hamiltonian"),
    "phi_wrap": ("const int k1 = (k + 1) % np;", "const int k1 = (k + 1 < np) ? k + 1 : k;",
                 "test_phi_periodic_wrap"),
    "kappa_prefactor": ("return 9.78e-3 * ne * ne * G", "return 8.78e-3 * ne * ne * G",
                        "test_kappa_matches_classical_free_free"),
    "gaunt_hot_constant": ("(24.5 + lnT - std::log(f))", "(25.5 + lnT - std::log(f))",
                           "test_kappa_matches_classical_free_free"),
}


def _build_and_run(name, tmp):
    orig, bad, pin = MUTANTS[name]
    src = open(SRC).read()
    assert orig in src, name
    d = os.path.join(tmp, name)
    os.makedirs(d)
    for f in ("rt_oracle.h", "ad_tape.h"):
        shutil.copy(os.path.join(ROOT, "oracle", f), d)
    with open(os.path.join(d, "rt_oracle.cpp"), "w") as fh:
        fh.write(src.replace(orig, bad, 1))
    so = os.path.join(d, "liborc.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", so,
                           os.path.join(d, "rt_oracle.cpp")])
    env = dict(os.environ, RT_ORACLE_LIB=so, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py") + "::" + pin],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    return name, r.returncode


def test_pins_catch_planted_mistakes(tmp_path):
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(lambda n: _build_and_run(n, str(tmp_path)), MUTANTS))
    survivors = [n for n, rc in results if rc == 0]
    assert not survivors, f"pins missed planted mistakes: {survivors}"
    assert all(rc == 1 for _, rc in results), results  # 1 = a test failed (not a crash)
