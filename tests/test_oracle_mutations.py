"""The oracle's pins catch plausible mistakes.

Each case plants one small mistake in a copy of oracle/glbe_oracle.c or
oracle/glbe_oracle2d.c (a dropped term, a wrong sign, index or factor, a
transposed operand), builds it in a temporary directory, and runs the pin
suite (tests/test_oracle_pins.py, or tests/test_oracle2d_pins.py for the 2D
oracle) against it in a subprocess: the pins named for that mistake must
fail.  The unmodified source must pass (checked once, so that a failure here means the pins, not the harness,
caught the mistake).  Everything runs on the CPU.
"""
import os
import subprocess
import sys

import pytest

pytest.importorskip("pytest_timeout")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "glbe_oracle.c")
SRC2D = os.path.join(ROOT, "oracle", "glbe_oracle2d.c")

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
    ("bounce-back into the same slot", "fn[n*19 + opp19[a]] = ft[a] - wall;", "fn[n*19 + a] = ft[a] - wall;",
     "poiseuille_exact or mrt_with_equal_rates"),
    ("anti-bounce-back sign", "gn[n*21 + j*7 + opp7[a]] = -gt[j*7+a] + 2.0*W7(a)*p->B0[j];",
     "gn[n*21 + j*7 + opp7[a]] = gt[j*7+a];", "hartmann_profile"),
    ("residual squares dropped", "num += du*du;", "num += fabs(du);", "residual_definition"),
]


# the same for the D2Q9 + D2Q5 oracle
MUTATIONS_2D = [
    ("2D equilibrium energy loses 1/gamma", "meq[1] = -2.0*rho + 3.0*jj/(gamma*rho);",
     "meq[1] = -2.0*rho + 3.0*jj/rho;", "equilibrium_moments"),
    ("2D equilibrium p_xy takes j_x twice", "meq[8] = j[0]*j[1]/(gamma*rho);", "meq[8] = j[0]*j[0]/(gamma*rho);",
     "equilibrium_moments"),
    ("2D source row 7 loses its factor 2", "S[7] = 2.0*(F[0]*u[0] - F[1]*u[1]);", "S[7] = (F[0]*u[0] - F[1]*u[1]);",
     "source"),
    ("2D P_S row 1 gets 1/gamma", "const double d[9] = {1.0, ig2, ig2, ig, ig, ig, ig, ig2, ig2};",
     "const double d[9] = {1.0, ig, ig2, ig, ig, ig, ig, ig2, ig2};", "source"),
    ("2D viscous rate ignores gamma", "const double snu = 1.0/(3.0*p->nu/p->gamma + 0.5);",
     "const double snu = 1.0/(3.0*p->nu + 0.5);", "relaxation_rates or mrt_with_equal_rates"),
    ("2D tau_m ignores gamma_m", "return p->eta/(p->gamma_m*THETA2) + 0.5;", "return p->eta/THETA2 + 0.5;",
     "induction_diffusion or d2q5"),
    ("2D D2Q5 weights of D2Q4-plus-rest", "return a == 0 ? 1.0/3.0 : 1.0/6.0;", "return a == 0 ? 0.2 : 0.2;",
     "d2q5 or induction_diffusion"),
    ("2D half force doubled", "jv[d] = m[d] + 0.5*F[d]/gam;", "jv[d] = m[d] + F[d]/gam;",
     "uniform_forcing or mrt_with_equal_rates"),
    ("2D current density sign", "return -c*(L[0][1] - L[1][0]);", "return c*(L[0][1] - L[1][0]);",
     "current_density"),
    ("2D Lorentz force sign", "FL[0] = -Jz*B[1];", "FL[0] = Jz*B[1];", "hartmann_profile or lorentz"),
    ("2D bounce-back into the same slot", "if (solid2(p, xt, yt)) fn[n*9 + opp9(a)] = ft[a];",
     "if (solid2(p, xt, yt)) fn[n*9 + a] = ft[a];", "poiseuille_exact or mrt_with_equal_rates"),
    ("2D anti-bounce-back sign", "if (sol) gn[n*10 + j*5 + opp5(a)] = -gt[j*5+a] + 2.0*W5(a)*p->B0[j];",
     "if (sol) gn[n*10 + j*5 + opp5(a)] = gt[j*5+a];", "hartmann_profile"),
    ("2D residual squares dropped", "num += du*du;", "num += fabs(du);", "residual_definition"),
]


def _run_pins(tmp_path, source_text, select=None, two_d=False):
    d = tmp_path / "oracle_variant"
    d.mkdir(exist_ok=True)
    src = d / ("glbe_oracle2d.c" if two_d else "glbe_oracle.c")
    src.write_text(source_text)
    env = dict(os.environ, GLBE_ORACLE_BUILD_DIR=str(d / "_build"))
    env["GLBE_ORACLE2D_SOURCE" if two_d else "GLBE_ORACLE_SOURCE"] = str(src)
    pins = "test_oracle2d_pins.py" if two_d else "test_oracle_pins.py"
    # a pin that no longer converges fails on the per-test time limit
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins), "-x", "-q",
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


def test_unmodified_2d_copy_passes(tmp_path):
    code, out = _run_pins(tmp_path, open(SRC2D).read(), two_d=True)
    assert code == 0, out


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS_2D, ids=[m[0] for m in MUTATIONS_2D])
def test_2d_pins_catch_the_mistake(tmp_path, name, old, new, pins):
    text = open(SRC2D).read()
    assert text.count(old) == 1, f"mutation site not found once: {old}"
    code, out = _run_pins(tmp_path, text.replace(old, new), pins, two_d=True)
    assert code == 1, f"the pins '{pins}' did not fail for: {name}\n{out}"
