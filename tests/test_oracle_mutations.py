"""Plants plausible mistakes in a copy of the oracle (CPU only) and checks
that the pins in test_oracle_pins.py catch every one of them.

The Philox round structure is deliberately absent: it is pinned only
statistically, so its parity with the published generator is unpinned.
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
    ("orc_transmitter(V[j],", "orc_transmitter(V[i],"),                    # index
    ("m[i] * m[i] * m[i] * h[i]", "m[i] * m[i] * h[i]"),                   # exponent
    ("double iL = p[P_GL] * (V[i] - p[P_EL]);", "double iL = 0.0;"),       # dropped term
    ("s[k] * s[k] * s[k] * s[k];", "s[k] * s[k] * s[k];"),                 # exponent
    ("- q[Q_K4] * s[k];", "- q[Q_K3] * s[k];"),                            # operand
    ("exp(-(V + 65.0) / 18.0)", "exp(-(V + 65.0) / 20.0)"),                # constant
    ("dh[i] = a[2] * (1.0 - h[i]) - a[3] * h[i];",
     "dh[i] = a[3] * (1.0 - h[i]) - a[2] * h[i];"),                        # swapped
    ("step < net->pulse_off[i]", "step <= net->pulse_off[i]"),             # off by one
    ("- iKL - isyn) / p[P_C];", "- iKL + isyn) / p[P_C];"),                # sign
    ("(V[i] - p[P_EKL])", "(V[i] - p[P_EK])"),                             # operand
    ("/ p[P_C];", ";"),                                                    # dropped factor
    ("(iext[i] - iNa", "(- iNa"),                                          # dropped input
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
                        "tests/test_oracle_pins.py"], cwd=tmp_path, capture_output=True, text=True)
    assert r.returncode != 0, "mutant survived: " + new + "\n" + r.stdout[-400:]
