"""Planted mistakes in a copy of the oracle must fail its CPU pins.

Each mutant is one plausible error in one step of the method -- a dropped term, a
wrong sign, a swapped ratio, a wrong exponent -- made in a temporary copy of
``oracle/`` (the committed oracle is never touched).  The copy is built by its own
loader with the same compiler flags, then the pin tests -- ``tests/test_oracle_pins.py``
(all but the 18 s vortex study) for the scheme, ``tests/test_oracle_learned.py`` for
the learned path -- run against it in a subprocess whose ``import oracle`` resolves to
the copy.  The unmodified copy must pass; every mutant must make at least one pin
fail.  This shows that the pins fix the oracle from outside itself: none of them
merely re-evaluates the oracle's own formula.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (what is wrong, file, original line fragment, planted line fragment)
MUTANTS = [
    ("piece rule: the 1/2 of the offset rounding dropped (Section 4.2)",
     "dvm_oracle.c", "long long num = 2 * k * n + p;", "long long num = 2 * k * n;"),
    ("Maxwellian: exponent -|v-u|^2/theta instead of /(2 theta) (Eq. M)",
     "dvm_oracle.c", "M[k] = pref * exp(-q / (2.0 * theta));", "M[k] = pref * exp(-q / theta);"),
    ("collision invariant |v|^2 instead of |v|^2 / 2 (Section 3)",
     "dvm_oracle.c", "m[d + 1] = 0.5 * v2;", "m[d + 1] = v2;"),
    ("relaxation factor exp(-tau/dt) instead of exp(-dt/tau) (Section 4.3.1)",
     "dvm_oracle.c", "S->lam[c] = exp(-S->dt / t);", "S->lam[c] = exp(-t / S->dt);"),
    ("HOFKS correction with U_M - U_E instead of U_E - U_M (Eq. minim_full)",
     "dvm_oracle.c", "r[i] = S->UE[i * nc + c] - um[i];", "r[i] = um[i] - S->UE[i * nc + c];"),
    ("MUSCL face flux with sigma+ + sigma- instead of sigma+ - sigma- (Eq. discmom)",
     "dvm_oracle.c", "0.25 * (sp - sm);", "0.25 * (sp + sm);"),
    ("flux splitting G+ = F - alpha U (Eq. discmom)",
     "dvm_oracle.c", "Gp[s] = Fs[s][i] + alpha * Us[s][i];", "Gp[s] = Fs[s][i] - alpha * Us[s][i];"),
    ("van Leer slope without its |a||b| term (Section 4.3.2)",
     "dvm_oracle.c", "return (fabs(a) * fabs(b) + a * b) / (a + b);", "return (a * b) / (a + b);"),
    ("exact Riemann solver: rarefaction density (p*/p)^gamma instead of ^(1/gamma)",
     "riemann.c", "*r = rl * pow(ps / pl, 1.0 / gamma);", "*r = rl * pow(ps / pl, gamma);"),
    ("network gradient: 1 + tanh^2 instead of the derivative 1 - tanh^2",
     "mlp.c", "d1[i] = s2 * (1.0 - h1[i] * h1[i]);", "d1[i] = s2 * (1.0 + h1[i] * h1[i]);"),
    ("network forward: second layer reads W2 transposed",
     "mlp.c", "s += W2[j * NH + i] * h1[i];", "s += W2[i * NH + j] * h1[i];"),
]

# the learned path: flagged step, non-equilibrium label, features
LEARNED_MUTANTS = [
    ("flagged cell keeps its lambda instead of the lambda -> 0 form (Theorem 1)",
     "dvm_oracle.c", "lam_eff[c] = fl ? 0.0 : S->lam[c];", "lam_eff[c] = S->lam[c];"),
    ("flagged cells not written back as E[U^{n+1}]",
     "dvm_oracle.c", "if (!(flags[c] != 0 && lam[c] != 1.0)) continue;", "if (1) continue;"),
    ("label normalised by ||f|| instead of ||E[U]||",
     "dvm_oracle.c", "den += fabs(E[k]);", "den += fabs(f[k * nc + c]);"),
    ("shear features with the derivatives transposed (d u_x/dx, d u_y/dy)",
     "dvm_oracle.c", "t * fabs(Dq[2][1]), t * fabs(Dq[3][0])", "t * fabs(Dq[2][0]), t * fabs(Dq[3][1])"),
    ("central difference over dx instead of 2 dx",
     "dvm_oracle.c", "const double h2 = 2.0 * g->dx;", "const double h2 = g->dx;"),
]


# the WENO Euler solver (Section 4.3.3), against tests/test_oracle_weno.py
WENO_MUTANTS = [
    ("WENO5 optimal weights in the wrong order (3/10, 6/10, 1/10)",
     "dvm_oracle.c", "const double d0 = 0.1, d1 = 0.6, d2 = 0.3;", "const double d0 = 0.3, d1 = 0.6, d2 = 0.1;"),
    ("WENO5 left candidate with 9 v_j instead of 11 v_j",
     "dvm_oracle.c", "(2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) / 6.0", "(2.0 * v[0] - 7.0 * v[1] + 9.0 * v[2]) / 6.0"),
    ("WENO5 smoothness indicator of the right stencil without its first-derivative term",
     "dvm_oracle.c", "13.0 / 12.0 * a2 * a2 + 0.25 * b2 * b2;", "13.0 / 12.0 * a2 * a2;"),
    ("WENO5 nonlinear weights d_k / (eps + beta_k) instead of its square",
     "dvm_oracle.c", "const double w1 = d1 / ((eps + beta1) * (eps + beta1));", "const double w1 = d1 / (eps + beta1);"),
    ("WENO f- reconstructed on the left-biased stencil (not mirrored)",
     "dvm_oracle.c", "fm[s] = 0.5 * (Fs[5 - s][i] - alpha * Us[5 - s][i]);",
     "fm[s] = 0.5 * (Fs[s + 1][i] - alpha * Us[s + 1][i]);"),
    ("WENO split flux f- = (F + alpha U)/2",
     "dvm_oracle.c", "fm[s] = 0.5 * (Fs[5 - s][i] - alpha * Us[5 - s][i]);",
     "fm[s] = 0.5 * (Fs[5 - s][i] + alpha * Us[5 - s][i]);"),
    ("SSP-RK3 second stage 1/2 W + 1/2 (...) instead of 3/4 and 1/4",
     "dvm_oracle.c", "W2[i] = 0.75 * W[i] + 0.25 * (W1[i] + dt * L[i]);", "W2[i] = 0.5 * W[i] + 0.5 * (W1[i] + dt * L[i]);"),
    ("SSP-RK3 last stage weights 1/2, 1/2 instead of 1/3, 2/3",
     "dvm_oracle.c", "Wout[i] = W[i] / 3.0 + 2.0 / 3.0 * (W2[i] + dt * L[i]);", "Wout[i] = W[i] / 2.0 + 1.0 / 2.0 * (W2[i] + dt * L[i]);"),
]


# the Strang splitting of FKS (Section 4.2), against tests/test_oracle_strang.py
STRANG_MUTANTS = [
    ("Strang half step with the full-step factor exp(-dt/tau)",
     "dvm_oracle.c", "S->lamh[c] = exp(-S->dt / (2.0 * t));", "S->lamh[c] = exp(-S->dt / t);"),
    ("Strang step without its first half relaxation",
     "dvm_oracle.c", "int rc = relax_half(S);", "int rc = 0;"),
    ("half relaxation with the weights swapped",
     "dvm_oracle.c", "S->f[k * nc + c] = l * S->f[k * nc + c] + (1.0 - l) * S->Eq[k * nc + c];",
     "S->f[k * nc + c] = (1.0 - l) * S->f[k * nc + c] + l * S->Eq[k * nc + c];"),
]


def oracle_copy(tmp_path, mutant=None):
    dst = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), dst,
                    ignore=shutil.ignore_patterns("*.so", "*.tmp*", "__pycache__"))
    if mutant is not None:
        _, fname, old, new = mutant
        path = dst / fname
        src = path.read_text()
        assert src.count(old) == 1, (fname, old)
        path.write_text(src.replace(old, new))
    return tmp_path


def run_in(tmp_path, args, timeout=300):
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT]))
    return subprocess.run([sys.executable] + args, cwd=str(tmp_path), env=env, capture_output=True,
                          text=True, timeout=timeout)


def pins_against(tmp_path, module="test_oracle_pins.py"):
    build = run_in(tmp_path, ["-c", "import oracle; oracle.build(force=True); print(oracle.__file__)"])
    assert build.returncode == 0, build.stderr[-2000:]
    assert build.stdout.strip().startswith(str(tmp_path)), build.stdout
    return run_in(tmp_path, ["-m", "pytest", os.path.join(ROOT, "tests", module), "-x", "-q",
                             "-p", "no:cacheprovider", "-k", "not isentropic_vortex"])


@pytest.mark.parametrize("module", ["test_oracle_pins.py", "test_oracle_learned.py", "test_oracle_weno.py",
                                    "test_oracle_strang.py"])
def test_unmodified_copy_passes_the_pins(tmp_path, module):
    r = pins_against(oracle_copy(tmp_path), module)
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0].split(":")[0][:40] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, mutant):
    r = pins_against(oracle_copy(tmp_path, mutant))
    assert r.returncode == 1 and " failed" in r.stdout, (mutant[0], r.returncode, r.stdout[-3000:])


@pytest.mark.parametrize("mutant", LEARNED_MUTANTS, ids=[m[0][:40] for m in LEARNED_MUTANTS])
def test_planted_mistake_in_the_learned_path_fails_a_pin(tmp_path, mutant):
    r = pins_against(oracle_copy(tmp_path, mutant), "test_oracle_learned.py")
    assert r.returncode == 1 and " failed" in r.stdout, (mutant[0], r.returncode, r.stdout[-3000:])


@pytest.mark.parametrize("mutant", WENO_MUTANTS, ids=[m[0][:40] for m in WENO_MUTANTS])
def test_planted_mistake_in_the_weno_solver_fails_a_pin(tmp_path, mutant):
    r = pins_against(oracle_copy(tmp_path, mutant), "test_oracle_weno.py")
    assert r.returncode == 1 and " failed" in r.stdout, (mutant[0], r.returncode, r.stdout[-3000:])


@pytest.mark.parametrize("mutant", STRANG_MUTANTS, ids=[m[0][:40] for m in STRANG_MUTANTS])
def test_planted_mistake_in_the_strang_splitting_fails_a_pin(tmp_path, mutant):
    r = pins_against(oracle_copy(tmp_path, mutant), "test_oracle_strang.py")
    assert r.returncode == 1 and " failed" in r.stdout, (mutant[0], r.returncode, r.stdout[-3000:])
