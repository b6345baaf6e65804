"""The oracle's pins catch plausible mistakes.

Each case plants one small mistake in a copy of oracle/glbe_oracle.c (a
dropped term, a wrong sign, index or factor, a transposed operand), builds it
in a temporary directory, and runs the pin suite (tests/test_oracle_pins.py)
against it in a subprocess: the pins named for that mistake must fail.  The unmodified source must
pass (checked once, so that a failure here means the pins, not the harness,
caught the mistake).  Everything runs on the CPU.
"""
import os
import subprocess
import sys

import pytest

pytest.importorskip("pytest_timeout")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "glbe_oracle.c")

# (name, exact text in glbe_oracle.c, replacement, the pins expected to catch it)
MUTATIONS = [
    ("equilibrium energy loses 1/gamma", "meq[1]  = -11.0*rho + 19.0*jj/gr;", "meq[1]  = -11.0*rho + 19.0*jj/rho;",
     "equilibrium_moments"),
    ("equilibrium p_xy takes j_z", "meq[13] = j[0]*j[1]/gr;", "meq[13] = j[0]*j[2]/gr;", "equilibrium_moments"),
    ("source row 9 loses its factor 2", "S[9]  = 2.0*(2.0*F[0]*u[0] - F[1]*u[1] - F[2]*u[2]);",
     "S[9]  = (2.0*F[0]*u[0] - F[1]*u[1] - F[2]*u[2]);", "source"),
    ("P_S row 1 gets 1/gamma", "PS[0] = 1.0; PS[1] = g2; PS[2] = g2;", "PS[0] = 1.0; PS[1] = g1; PS[2] = g2;",
     "source"),
    ("viscous rate ignores gamma", "double snu = 1.0 / (3.0*p->nu/p->gamma + 0.5);",
     "double snu = 1.0 / (3.0*p->nu + 0.5);", "relaxation_rates or mrt_with_equal_rates"),
    ("tau_m ignores gamma_m", "return p->eta / (p->gamma_m * THETA_M) + 0.5;", "return p->eta / THETA_M + 0.5;",
     "induction_diffusion"),
    ("half force doubled", "jv[d] = m[d] + 0.5*F[d]/gam;", "jv[d] = m[d] + F[d]/gam;",
     "uniform_forcing or mrt_with_equal_rates"),
    ("current density sign", "double coef = -1.0 / (p->mu * p->chi * orc_tau_m(p) * THETA_M);",
     "double coef = 1.0 / (p->mu * p->chi * orc_tau_m(p) * THETA_M);", "current_density"),
    ("Lorentz force operands transposed", "FL[0] = J[1]*B[2] - J[2]*B[1];", "FL[0] = J[2]*B[1] - J[1]*B[2];",
     "hartmann_profile"),
    ("bounce-back into the same slot", "fn[n*19 + opp19[a]] = ft[a];", "fn[n*19 + a] = ft[a];",
     "poiseuille_exact or mrt_with_equal_rates"),
    ("anti-bounce-back sign", "gn[n*21 + j*7 + opp7[a]] = -gt[j*7+a] + 2.0*W7(a)*p->B0[j];",
     "gn[n*21 + j*7 + opp7[a]] = gt[j*7+a];", "hartmann_profile"),
    ("residual squares dropped", "num += du*du;", "num += fabs(du);", "residual_definition"),
]


def _run_pins(tmp_path, source_text, select=None):
    d = tmp_path / "oracle_variant"
    d.mkdir(exist_ok=True)
    src = d / "glbe_oracle.c"
    src.write_text(source_text)
    env = dict(os.environ, GLBE_ORACLE_SOURCE=str(src), GLBE_ORACLE_BUILD_DIR=str(d / "_build"))
    # a pin that no longer converges fails on the per-test time limit
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x", "-q",
                        "-p", "no:cacheprovider", "--timeout", "60"] + (["-k", select] if select else []),
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-2000:]


def test_unmodified_copy_passes(tmp_path):
    code, out = _run_pins(tmp_path, open(SRC).read())
    assert code == 0, out


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_the_mistake(tmp_path, name, old, new, pins):
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site not found once: {old}"
    code, out = _run_pins(tmp_path, text.replace(old, new), pins)
    assert code == 1, f"the pins '{pins}' did not fail for: {name}\n{out}"   # 1: tests failed (5: none selected)
