"""The pins catch plausible mistakes: for each of a few one-line mistakes
planted in a copy of the oracle's C source (a wrong sign, a dropped factor, a
transposed index, a lost clip, a shifted centre, a tie-break), the copy is
compiled and the relevant pin files run against it in a subprocess; at least
one pin must fail.  The oracle itself is not modified."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fofse_oracle.c")
OUT = os.path.join(ROOT, "oracle", "_build", "mutants")
PINS = "tests/test_oracle_pins.py"
VOL = "tests/test_oracle_volume.py"
VOLADJ = "tests/test_oracle_volume_adjoint.py"
BADJ = "tests/test_oracle_batch_adjoint.py"

MUTATIONS = [
    ("projection-sign", "im -= rw[m * Ls + n] * s[p];", "im += rw[m * Ls + n] * s[p];", [PINS]),
    ("tie-break", "if (v > best) {", "if (v >= best) {", [PINS]),
    ("dropped-gamma", "double cr = gamma * P_re[ui] / W0;", "double cr = P_re[ui] / W0;", [PINS]),
    ("weight-centre", "double c = border + (block - 1) / 2.0;", "double c = border + block / 2.0;", [PINS]),
    ("adjoint-sign", "gbar[i] -= wL[i] * q[i];", "gbar[i] += wL[i] * q[i];", [PINS]),
    ("ofse-index", "int a = ((u1 - l1 + T) % T) * T + (u2 - l2 + T) % T;",
     "int a = ((l1 - u1 + T) % T) * T + (l2 - u2 + T) % T;", ["tests/test_oracle_ofse.py"]),
    ("dct-norm", "nrm += wL[m * Ls + n] * ph * ph;", "nrm += wL[m * Ls + n] * ph;",
     ["tests/test_oracle_dct.py"]),
    ("curve-clip", "v = v < 0.0 ? 0.0 : (v > 255.0 ? 255.0 : v);", "v = v < 0.0 ? 0.0 : v;",
     ["tests/test_oracle_curve.py"]),
    ("fd-conjugate", "ti += cr * W_im[b] - ci * W_re[b];", "ti += cr * W_im[b] + ci * W_re[b];", [PINS]),
    ("ofse-factor", "gr = W0 * (pr * q_re + pi * q_im) / den;", "gr = (pr * q_re + pi * q_im) / den;",
     ["tests/test_oracle_ofse.py"]),
    ("dct-energy-scale", "double e = P[i] * P[i] * (k1 ? 2.0 : 1.0) * (k2 ? 2.0 : 1.0);",
     "double e = P[i] * P[i];", ["tests/test_oracle_dct.py"]),
    ("volume-temporal-sign", "im += yi * ct[p] - yr * st[p];", "im += yi * ct[p] + yr * st[p];", [VOL]),
    ("volume-centre", "double dt = t - depth, dm = m - c, dn = n - c;",
     "double dt = t - depth - 1, dm = m - c, dn = n - c;", [VOL]),
    ("volume-B-every-frame", "int inB = t == depth && m >= border", "int inB = m >= border", [VOL]),
    ("volume-pair-weight", "(2 * u2) % T == 0 && (2 * u3) % Tt == 0) ? 0 : 1;",
     "(2 * u2) % T == 0) ? 0 : 1;", [VOL]),
    ("volume-canonical", "return lin3(k1, k2, k3, T, Tt) <= lin3(", "return lin3(k1, k2, k3, T, Tt) < lin3(",
     [VOL]),
    ("volume-tie-break", "if (e > top) {", "if (e >= top) {", [VOL]),
    ("volume-synthesis-phase", "(long)u[2] * tau * T) % M;", "(long)u[2] * tau) % M;", [VOL]),
    ("volume-adjoint-projection-sign", "double qv = pbar_re * cs[i] - pbar_im * sn[i];",
     "double qv = pbar_re * cs[i] + pbar_im * sn[i];", [VOLADJ]),
    ("volume-adjoint-model-sign", "gbar[i] -= wL[i] * qv;", "gbar[i] += wL[i] * qv;", [VOLADJ]),
    ("volume-fd-shift", "long a = lin3((k1 - u[0] + T) % T, (k2 - u[1] + T) % T, (k3 - u[2] + Tt) % Tt, T, Tt);",
     "long a = lin3((k1 - u[0] + T) % T, (k2 - u[1] + T) % T, (k3 + u[2]) % Tt, T, Tt);", [VOL]),
    ("batch-adjoint-plan-index", "grg[2 * bd[2]] += oracle_rho_chain(", "grg[0] += oracle_rho_chain(", [BADJ]),
    ("batch-adjoint-gamma-overwrite", "grg[2 * bd[2] + 1] += gam;", "grg[2 * bd[2] + 1] = gam;", [BADJ]),
    ("batch-adjoint-frame-overwrite", "gf[(size_t)fy * J->width + fx] += fbar[i];",
     "gf[(size_t)fy * J->width + fx] = fbar[i];", [BADJ]),
    ("batch-adjoint-thread-sum", "grad_frame[i] += J.grad_frame_t[t][i];",
     "grad_frame[i] = J.grad_frame_t[t][i];", [BADJ]),
]


@pytest.mark.parametrize("name,old,new,files", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(name, old, new, files):
    src = open(SRC).read()
    assert old in src, name
    os.makedirs(OUT, exist_ok=True)
    c = os.path.join(OUT, f"{name}.c")
    so = os.path.join(OUT, f"{name}.so")
    with open(c, "w") as f:
        f.write(src.replace(old, new, 1))
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-o", so, c, "-lm", "-lpthread"])
    env = dict(os.environ, FOFSE_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider", *files],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin failed for the planted mistake {name}:\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout, r.stdout[-2000:]
