"""Plants plausible mistakes in a private copy of the oracle's C source and
checks that the pins in test_oracle_pins.py (and test_oracle_pins_ext.py) catch every one of them (CPU only).

Each mutation is applied to a copy in a temporary directory, built there, and
the pin tests run in a subprocess against that copy; the committed oracle is
never touched."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PINS = "test_oracle_pins.py"
EXT = "test_oracle_pins_ext.py"

MUTATIONS = [
    ("PDG delta sign in U_e3", "U[0][2] = s13 * emid;", "U[0][2] = s13 * eid;"),
    ("matter sign not flipped for nubar", "M[0][0] += nubar ? -A_abs : A_abs;", "M[0][0] += A_abs;"),
    ("Hamiltonian transposed", "s += U[b][i] * m2[i] * conj(U[a][i]);", "s += U[a][i] * m2[i] * conj(U[b][i]);"),
    ("propagator phase sign", "ph[k] = cexp(-I * tau * lam[k]);", "ph[k] = cexp(I * tau * lam[k]);"),
    ("dm31 taken as dm32", "double m2[3] = {0.0, pt->dm21, pt->dm32 + pt->dm21};",
     "double m2[3] = {0.0, pt->dm21, pt->dm32};"),
    ("matter constant missing factor 2", "return 2.0 * V * 1e9;", "return V * 1e9;"),
    ("binning ignores lo", "float u = t * inv_f;", "float u = x * inv_f;"),
    ("nubar keeps U", "for (int i = 0; i < 3; ++i) U[a][i] = conj(U[a][i]);",
     "for (int i = 0; i < 3; ++i) U[a][i] = U[a][i];"),
    ("weight drops norm", "return p * (double)w_mc * pt->norm;", "return p * (double)w_mc;"),
    ("Jacobi rotation missing its phase", "G[q][q] = c * emphi;", "G[q][q] = c;"),
    ("propagator built from conjugated eigenvectors", "s += V[b][k] * ph[k] * conj(V[a][k]);",
     "s += conj(V[b][k]) * ph[k] * V[a][k];"),
    ("bin centre without the half", "double c = t_lo + ((double)t + 0.5) * w;", "double c = t_lo + (double)t * w;",
     EXT),
    ("binned method uses the event energy", "p = orc_prob(pt, L_km, rho, ye, (double)orc_true_centre(t_lo, t_hi, t_nbins, t),",
     "p = orc_prob(pt, L_km, rho, ye, (double)e_true[i] + 0.0 * t,", EXT),
    ("binned method keeps events below the range", "if (t >= 0)\n            p = orc_prob",
     "if (t >= -1)\n            p = orc_prob", EXT),
    ("reweight swaps initial and final flavour", "(double)e_true[i], flav_in[i], flav_out[i],",
     "(double)e_true[i], flav_out[i], flav_in[i],"),
    ("histogram ignores the point's energy scale", "scratch_w, pts[p].escale, lo, hi, nbins, compensated,",
     "scratch_w, pts[0].escale, lo, hi, nbins, compensated,"),
    ("histogram rows written at the wrong offset", "out + (int64_t)p * nbins);", "out + (int64_t)0 * nbins);"),
    ("histogram weights every point with the first point", "ye, &pts[p], 0,\n                     scratch_w);",
     "ye, &pts[0], 0,\n                     scratch_w);"),
    ("layers multiplied against the order of travel", "mat_mul(Sk, S, S);", "mat_mul(S, Sk, S);", EXT),
    ("every layer at the first layer's density", "orc_matter_A(rho[k], ye[k], E_GeV)",
     "orc_matter_A(rho[0], ye[0], E_GeV)", EXT),
    ("layer phase uses the total length", "orc_evolution(M, orc_c_L() * L_km[k] / E_GeV, Sk);",
     "orc_evolution(M, orc_c_L() * L_km[0] / E_GeV, Sk);", EXT),
]


@pytest.mark.parametrize("name,old,new,pins", [m if len(m) == 4 else m + (PINS,) for m in MUTATIONS],
                         ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new, pins):
    src = open(os.path.join(ROOT, "oracle", "osc_oracle.c")).read()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), pkg / "__init__.py")
    (pkg / "osc_oracle.c").write_text(src.replace(old, new))
    env = dict(os.environ, PYTHONPATH=str(tmp_path) + os.pathsep + ROOT)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins),
                        "-q", "-x", "-p", "no:cacheprovider", "--rootdir", str(tmp_path)],
                       cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, "planted mistake '%s' not caught:\n%s" % (name, r.stdout[-2000:])
