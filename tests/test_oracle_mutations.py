"""Plants plausible mistakes in a copy of the oracle (CPU only) and checks
that the pins in test_oracle_pins.py, test_oracle_adjoint.py and
test_oracle_tableau.py catch every one of them.

The Philox mutants are caught by the generator's published known-answer
vectors (tests/golden/philox_kat.json).
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = [
    ("2.0 * k3[i] + k4[i]", "1.0 * k3[i] + k4[i]"),                       # RK4 weight
    ("Y[i] = y[i] + h * k3[i];", "Y[i] = y[i] + 0.5 * h * k3[i];"),        # RK4 node
    ("- q[Q_B] * r[k];", "+ q[Q_B] * r[k];"),                              # sign
    ("G * (V[i] - q[Q_E]);", "G * (V[j] - q[Q_E]);"),                      # index
    ("double T = orc_transmitter(V[j], q[Q_VP]", "double T = orc_transmitter(V[i], q[Q_VP]"),  # index
    ("double iNa = p[P_GNA] * m[i] * m[i] * m[i] * h[i]", "double iNa = p[P_GNA] * m[i] * m[i] * h[i]"),  # exponent
    ("double iL = p[P_GL] * (V[i] - p[P_EL]);", "double iL = 0.0;"),       # dropped term
    ("s[k] * s[k] * s[k] * s[k];\n                G = s4 / (s4 + q[Q_KD]);",
     "s[k] * s[k] * s[k];\n                G = s4 / (s4 + q[Q_KD]);"),                  # exponent
    ("- q[Q_K4] * s[k];", "- q[Q_K3] * s[k];"),                            # operand
    ("exp(-(V + 65.0) / 18.0)", "exp(-(V + 65.0) / 20.0)"),                # constant
    ("dh[i] = a[2] * (1.0 - h[i]) - a[3] * h[i];",
     "dh[i] = a[3] * (1.0 - h[i]) - a[2] * h[i];"),                        # swapped
    ("step < net->pulse_off[i]", "step <= net->pulse_off[i]"),             # off by one
    ("- iKL - isyn) / p[P_C];", "- iKL + isyn) / p[P_C];"),                # sign
    ("double iKL = p[P_GKL] * (V[i] - p[P_EKL]);", "double iKL = p[P_GKL] * (V[i] - p[P_EK]);"),  # operand
    ("- iKL - isyn) / p[P_C];", "- iKL - isyn);"),                         # dropped factor
    ("(iext[i] - iNa", "(- iNa"),                                          # dropped input
    # discrete adjoint
    ("kb[i] = hstep / 3.0 * lam[i] + hstep * Yb[i];",
     "kb[i] = hstep / 3.0 * lam[i] + 0.5 * hstep * Yb[i];"),               # tableau transpose
    ("lam[i] += Ysum[i] + Yb[i];", "lam[i] += Ysum[i];"),                  # dropped stage
    ("uV[i] += q * (-diion - gsum);", "uV[i] += q * (-diion);"),           # dropped term
    ("uV[j] += vr[k] * sq[Q_A] * dT * (1.0 - r[k]);",
     "uV[i] += vr[k] * sq[Q_A] * dT * (1.0 - r[k]);"),                     # wrong index
    ("out[3] = r[3] * (1.0 - r[3]) / 10.0;", "out[3] = r[3] * (1.0 - r[3]) / 20.0;"),  # constant
    ("gp[P_GK] += -q * n4 * (V[i] - p[P_EK]);", "gp[P_GK] += q * n4 * (V[i] - p[P_EK]);"),  # sign
    ("if (g) g->gw[k] += -q * G * (V[i] - E);", "if (g) g->gw[k] += -q * (V[i] - E);"),  # dropped factor
    # forward Euler and its adjoint
    ("for (int64_t i = 0; i < d; ++i) y[i] = y[i] + h * work[i];",
     "for (int64_t i = 0; i < d; ++i) y[i] = y[i] + 0.5 * h * work[i];"),   # step size
    ("for (int64_t i = 0; i < d; ++i) kb[i] = hstep * lam[i];",
     "for (int64_t i = 0; i < d; ++i) kb[i] = lam[i];"),                    # dropped factor
    # tableau map and its adjoint
    ("Y[i] = y[i] + h * tab[st - 1] * k[i];", "Y[i] = y[i] + h * tab[st] * k[i];"),  # coefficient index
    ("sum[i] += tab[3 + st] * k[i];", "sum[i] += k[i];"),                  # dropped weight
    ("if (st < ns) kb[i] += hstep * tab[st] * Yb[i];",
     "if (st < ns) kb[i] += hstep * tab[st - 1] * Yb[i];"),                # coupling index
    ("kb[i] = hstep * tab[3 + st] * lam[i];", "kb[i] = hstep * lam[i];"),  # dropped weight
    ("Ys[(st - 1) * d + i] = y[i] + hstep * tab[st - 1] * k[i];",
     "Ys[(st - 1) * d + i] = y[i] + hstep * k[i];"),                       # dropped coefficient
    # Philox4x32-10
    ("const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;",
     "const uint32_t M0 = 0xCD9E8D57u, M1 = 0xD2511F53u;"),                # swapped multipliers
    ("if (round > 0) { k0 += W0; k1 += W1; }", "if (round > 0) { k0 += W0; }"),  # dropped key bump
    ("uint32_t n2 = hi0 ^ c3 ^ k1;", "uint32_t n2 = hi0 ^ c1 ^ k1;"),      # wrong word
    ("for (int round = 0; round < 10; ++round) {\n        if (round > 0) { k0",
     "for (int round = 0; round < 9; ++round) {\n        if (round > 0) { k0"),  # rounds
]


@pytest.mark.parametrize("old,new", MUTANTS)
def test_pins_catch_planted_mistake(tmp_path, old, new):
    for d in ("oracle", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("_build", "__pycache__"))
    pkg = tmp_path / "paper_1906_03958_gb300"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_1906_03958_gb300", "netgen.py"), pkg)
    (pkg / "__init__.py").write_text("")
    src = tmp_path / "oracle" / "psst_oracle.c"
    text = src.read_text()
    assert text.count(old) == 1, old
    src.write_text(text.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py", "tests/test_oracle_adjoint.py",
                        "tests/test_oracle_tableau.py"],
                       cwd=tmp_path, capture_output=True, text=True)
    assert r.returncode != 0, "mutant survived: " + new + "\n" + r.stdout[-400:]
