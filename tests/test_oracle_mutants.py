"""The oracle's pins catch plausible mistakes. Each mutant below plants one in a copy of the
oracle's C source (a dropped term, a wrong sign, index or operand, a transposed component),
builds it, and runs the pin files against it: every mutant must fail at least one pin.
The mistakes are planted in the oracle only, on the CPU."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE = os.path.join(ROOT, "oracle")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_window.py", "tests/test_oracle_smoothing.py",
        "tests/test_oracle_alm.py", "tests/test_oracle_scf.py", "tests/test_oracle_diagnostics.py"]

# (name, text in m2m_oracle.c, its replacement)
MUTANTS = [
    ("hernquist potential: wrong sign of a", "double phi = -p->G * p->M / (r + p->a);",
     "double phi = -p->G * p->M / (r - p->a);"),
    ("nfw potential: log instead of log1p", "phi += -p->G * p->Ms * log1p(r / p->rs) / r;",
     "phi += -p->G * p->Ms * log(r / p->rs) / r;"),
    ("log potential force: dropped flattening", "        *az = -v2 * z / (q2 * D);", "        *az = -v2 * z / D;"),
    ("hernquist force: dropped term", "double g = p->G * p->M / ((r + p->a) * (r + p->a));",
     "double g = p->G * p->M / ((r + p->a) * r);"),
    ("force: transposed component", "*ay = -g * y / r;", "*ay = -g * x / r;"),
    ("drift: transposed velocity", "s->x[i] += dt * s->vx[i];", "s->x[i] += dt * s->vy[i];"),
    ("hermite: sign of the alternating sum", "s += (m % 2 == 0) ? t : -t;", "s += t;"),
    ("gauss-hermite: normalisation index", "double norm = 1.0 / sqrt(pow(2.0, n + 1) * OR_PI * nfact);",
     "double norm = 1.0 / sqrt(pow(2.0, n) * OR_PI * nfact);"),
    ("projection: sign of the z term", "*Y = y * ci - z * si;", "*Y = y * ci + z * si;"),
    ("line of sight: sin and cos swapped", "*vlos = vy * si + vz * ci;", "*vlos = vy * ci + vz * si;"),
    ("entropy: sign of the log", "double dS = what_i > 0.0 ? -log(w_i / what_i) : 0.0;",
     "double dS = what_i > 0.0 ? log(w_i / what_i) : 0.0;"),
    ("global entropy: sign of the constant", "if (mode == OR_GWR) dS -= 1.0;", "if (mode == OR_GWR) dS += 1.0;"),
    ("force of change: sign of the data term", "return par->mu * dS - data;", "return par->mu * dS + data;"),
    ("temporal smoothing: dropped", "for (int j = 0; j < J; ++j) st->ytil[j] += par->alpha * (st->yraw[j] - st->ytil[j]);",
     "for (int j = 0; j < J; ++j) st->ytil[j] = st->yraw[j];"),
    ("residual: divided by sigma squared", "st->delta[j] = (st->ytil[j] - Y[j]) / sig[j];",
     "st->delta[j] = (st->ytil[j] - Y[j]) / (sig[j] * sig[j]);"),
    ("renormalisation: inverted", "for (long i = 0; i < s->n; ++i) s->w[i] *= st->W0 / W;",
     "for (long i = 0; i < s->n; ++i) s->w[i] *= W / st->W0;"),
    ("energy: kinetic term halved twice", "double E = 0.5 * (vx * vx + vy * vy + vz * vz) + or_phi(p, x, y, z);",
     "double E = 0.25 * (vx * vx + vy * vy + vz * vz) + or_phi(p, x, y, z);"),
    ("angular momentum: transposed component", "double Lx = y * vz - z * vy, Ly = z * vx - x * vz, Lz = x * vy - y * vx;",
     "double Lx = y * vz - z * vy, Ly = z * vx - x * vz, Lz = x * vx - y * vy;"),
    ("window: the upper edge left out", "for (int k2 = k - hE; k2 <= k + hE; ++k2)",
     "for (int k2 = k - hE; k2 < k + hE; ++k2)"),
    ("window: cells counted instead of particles", "nc += count[k2 * nx + l2];", "nc += 1;"),
    ("self-consistent potential: inner shell power", "                f = pow(r, l) / pow(rk, l + 1);",
     "                f = pow(r, l + 1) / pow(rk, l + 1);"),
    ("self-consistent potential: outer radial derivative sign", "df = -(l + 1) * pow(rk, l) / pow(r, l + 2);",
     "df = (l + 1) * pow(rk, l) / pow(r, l + 2);"),
    ("self-consistent potential: multipole constant", "double C = -4.0 * OR_PI * p->G / (2.0 * l + 1.0);",
     "double C = -4.0 * OR_PI * p->G / (2.0 * l - 1.0);"),
    ("cloud in cell: weights swapped", "g0 = (p->scf_r[k0 + 1] - r) / d;", "g0 = (r - p->scf_r[k0]) / d;"),
    ("smoothing: penalty sign", "for (size_t q = 0; q < (size_t)n * n; ++q) M[q] = lambda * P[q];",
     "for (size_t q = 0; q < (size_t)n * n; ++q) M[q] = -lambda * P[q];"),
    ("delta_grid: relative to the model", "double r = (wt - wm) / wt;", "double r = (wt - wm) / wm;"),
    ("kinematic sums: second moment linear", "o[4 + c] += w * v[c] * v[c];", "o[4 + c] += w * v[c];"),
    ("associated legendre: recurrence index", "double p2 = (x * (2.0 * ll - 1.0) * p1 - (ll + am - 1.0) * p0) / (ll - am);",
     "double p2 = (x * (2.0 * ll - 1.0) * p1 - (ll + am) * p0) / (ll - am);"),
    ("real harmonics: cos and sin swapped", "if (m > 0) return sqrt(2.0) * N * plm * cos(am * phi);",
     "if (m > 0) return sqrt(2.0) * N * plm * sin(am * phi);"),
    ("shell cloud in cell: weight of the outer point", "g_out[1] = (r - e[k - 1]) / d;", "g_out[1] = (e[k] - r) / d;"),
    ("target fit: sign of the V_p correction", "V[p] += sqrt(2.0) * s_old * h1;", "V[p] -= sqrt(2.0) * s_old * h1;"),
    ("circular orbit: L from v_c^2", "return R * sqrt(vc2);", "return R * vc2;"),
    ("circularity: not normalised", "double xc = (Lc > 0.0) ? L / Lc : 0.0;", "double xc = (Lc > 0.0) ? L : 0.0;"),
]


def _run(mutant, tmp):
    name, old, new = mutant
    src = open(os.path.join(ORACLE, "m2m_oracle.c")).read()
    assert src.count(old) == 1, name
    d = os.path.join(tmp, str(MUTANTS.index(mutant)))
    os.makedirs(d)
    with open(os.path.join(d, "m2m_oracle.c"), "w") as f:
        f.write(src.replace(old, new))
    shutil.copy(os.path.join(ORACLE, "m2m_oracle.h"), d)
    so = os.path.join(d, "liboracle.so")
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-o", so,
                    os.path.join(d, "m2m_oracle.c"), "-lm"], check=True)
    env = dict(os.environ, M2M_ORACLE_SO=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"] + PINS,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode


def test_every_planted_mistake_fails_a_pin():
    shutil.which("gcc") or pytest.skip("gcc is needed")
    with tempfile.TemporaryDirectory() as tmp, cf.ThreadPoolExecutor(4) as ex:
        results = list(ex.map(lambda m: _run(m, tmp), MUTANTS))
    survivors = [name for name, rc in results if rc == 0]
    assert not survivors, f"mutants no pin catches: {survivors}"
