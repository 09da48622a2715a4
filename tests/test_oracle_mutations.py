"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a private copy of oracle/maclab_oracle.c,
compiles it, and runs the oracle pin tests against that build in a child
process: every mutant must make at least one pin fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "maclab_oracle.c")

MUTANTS = {
    "bed_sign": ("bed = -(g * hbar", "bed = +(g * hbar"),
    "hbar_one_sided": ("hbar = 0.5 * (h[x] + h[s]);", "hbar = h[x];"),
    "force_not_centred": ("Fbar_x = 0.5 * (Fx[0] + sx * Fs[0]);", "Fbar_x = Fs[0];"),
    "bounce_same_dir": ("fa = fx[opposite(a)];", "fa = fx[a];"),
    "C_swapped": ("(a % 2 == 1) ? 1.0 / 3.0 : 1.0 / 12.0", "(a % 2 == 0) ? 1.0 / 3.0 : 1.0 / 12.0"),
    "lambda_swapped": ("(a % 2 == 1) ? 1.0 : 0.25", "(a % 2 == 0) ? 1.0 : 0.25"),
    "feq_drop_quadratic": ("eu * eu / (2.0 * e * e * e * e)", "0.0"),
    "feq0_coefficient": ("5.0 * g * h / (6.0 * e * e)", "4.0 * g * h / (6.0 * e * e)"),
    "specular_no_flip": ("*sy = -1;", "*sy = 1;"),
    "mirror_direction": ("CX[b] == sx * CX[a]", "CX[b] == CX[a]"),
    "push_instead_of_pull": ("int ii = i - CX[a], jj = j - CY[a];",
                             "int ii = i + CX[a], jj = j + CY[a];"),
    "friction_sign": ("- tbx / p->rho_w", "+ tbx / p->rho_w"),
    "coriolis_sign": ("- p->Omega * h * u;", "+ p->Omega * h * u;"),
    "force_weight": ("force = (dt / (e * e))", "force = (dt / e)"),
    "momentum_component": ("Shu += ex * fa;", "Shu += ey * fa;"),
    "dirichlet_old_level": ("u1[x] = u1[n1];", "u1[x] = u[n1];"),
    "dirichlet_linear": ("h1[x] = h1[n1];", "h1[x] = 2.0 * h1[n1] - h1[(size_t)(j + 2 * dj) * nx + (i + 2 * di)];"),
    "dirichlet_time_level": ("h1[x] = wave(p->bc[ed][0], t_next);\n                u1",
                             "h1[x] = wave(p->bc[ed][0], t_next - dx_dt_guard);\n                u1"),
    "noslip_missing": ("                u1[x] = 0.0;\n                v1[x] = 0.0;\n            }\n        }\n    }",
                       "            }\n        }\n    }"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation anchor not found: %s" % name
    mutated = src.replace(old, new, 1)
    if "dx_dt_guard" in new:
        mutated = mutated.replace("const double e = p->e, g = p->g, dt = p->dx / p->e;",
                                  "const double e = p->e, g = p->g, dt = p->dx / p->e;"
                                  " const double dx_dt_guard = dt;", 1)
    csrc = tmp_path / "mut.c"
    csrc.write_text(mutated)
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                           "-o", str(lib), str(csrc), "-lm"])
    env = dict(os.environ, ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "mutant %s survived the pins:\n%s" % (name, r.stdout[-2000:])
