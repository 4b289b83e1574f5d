"""The oracle's pins catch plausible mistakes: each case below plants one
mistake in a copy of oracle/dust_oracle.c (a dropped term, a wrong sign, a
wrong index or factor), builds it, and runs the pin suites against it; at
least one pin must fail.  Everything runs on the CPU."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dust_oracle.c")
PIN_SUITES = [os.path.join(ROOT, "tests", "test_oracle_weights.py"),
              os.path.join(ROOT, "tests", "test_oracle_push.py"),
              os.path.join(ROOT, "tests", "test_oracle_drag_work.py"),
              os.path.join(ROOT, "tests", "test_oracle_fixed_point.py")]

# (name, original text, planted text); the original must occur exactly once
MUTATIONS = [
    ("cartesian TSC centre weight", "w[1] = 0.75 - d * d;", "w[1] = 0.7 - d * d;"),
    ("cylindrical TSC outer factor", "w[2] = (d + 3.0 * nu + 2.0) / den",
     "w[2] = (d + 3.0 * nu + 1.0) / den"),
    ("theta-CIC lower weight sign", "w[0] = -(cos(lo) - cos(lo + d)) / D;",
     "w[0] = (cos(lo) - cos(lo + d)) / D;"),
    ("zone location not half-open", "if (edges[mid] <= x) lo = mid;",
     "if (edges[mid] < x) lo = mid;"),
    ("drag term with h1 instead of c_g", "pp[d] = E * pn[d] + cg * vg[d];",
     "pp[d] = E * pn[d] + h1 * vg[d];"),
    ("h1 dropped to dt E", "double h1 = (x == 0.0) ? dt : dt * cg / x;", "double h1 = dt * E;"),
    ("orbital-advection Omega2 without (1 - q/2)", "double Om2 = Om1 * (1.0 - 0.5 * qq);",
     "double Om2 = Om1;"),
    ("standard-frame Coriolis sign", "double G1 = -2.0 * (0.5 * pn[0]) * Om;",
     "double G1 = 2.0 * (0.5 * pn[0]) * Om;"),
    ("cylindrical l^2 not averaged", "double l2 = 0.5 * (pn[1] * pn[1] + pp[1] * pp[1]);",
     "double l2 = pn[1] * pn[1];"),
    ("spherical second square repeats l_phi",
     "double ar = lt2 / (r * r * r) + lp2 / (r * r * r * st * st) + g[0];",
     "double ar = lp2 / (r * r * r) + lp2 / (r * r * r * st * st) + g[0];"),
    ("second drift with end-point radius",
     "        q[1] = q[1] + h * p[1] / (qm[0] * qm[0]);\n        q[2] = q[2] + h * p[2];\n        break;",
     "        q[1] = q[1] + h * p[1] / (q[0] * q[0]);\n        q[2] = q[2] + h * p[2];\n        break;"),
    ("Stokes-number stopping time exponent", "return value * sqrt(R * R * R / P->gm);",
     "return value * sqrt(R * R / P->gm);"),
    ("energy channel with p^n", "D[3] += D[c] * dHdp[c];", "D[3] += D[c] * pn[c];"),
    ("cylindrical energy channel with l / R", "dHdp[1] = 0.5 * (pn[1] + pp[1]) / (R * R);",
     "dHdp[1] = 0.5 * (pn[1] + pp[1]) / R;"),
    ("spherical energy channel without sin^2 theta",
     "dHdp[2] = 0.5 * (pn[2] + pp[2]) / (r * r * st * st);", "dHdp[2] = 0.5 * (pn[2] + pp[2]) / (r * r);"),
    ("cylindrical energy channel with the end-point v_R",
     "dHdp[0] = 0.5 * (pn[0] + pp[0]);\n            dHdp[1] = 0.5 * (pn[1] + pp[1]) / (R * R);",
     "dHdp[0] = pp[0];\n            dHdp[1] = 0.5 * (pn[1] + pp[1]) / (R * R);"),
    ("shear-periodic y shift sign at +x", "if (q[0] >= hi) {\n                q[1] += shift;",
     "if (q[0] >= hi) {\n                q[1] -= shift;"),
    ("standard-frame v_y jump sign at +x", "if (!P->fargo) p[1] += P->q * P->omega * Lx;",
     "if (!P->fargo) p[1] -= P->q * P->omega * Lx;"),
    ("shear-periodic shift at the step's start time", "int alive = apply_bc(P, qn, pnew, t + dt);",
     "int alive = apply_bc(P, qn, pnew, t);"),
    ("deposit sign", "D[c] = -m * ((pp[c] - pn[c]) - dt * a[c]);",
     "D[c] = m * ((pp[c] - pn[c]) - dt * a[c]);"),
    ("cylindrical zone volume", "dV = 0.5 * (a1 * a1 - a0 * a0) * (b1 - b0) * (c1 - c0);",
     "dV = (a1 - a0) * (b1 - b0) * (c1 - c0);"),
    ("semi-implicit drag factor b = dt / tau", "double b = 0.5 * dt * it;", "double b = dt * it;"),
    ("predictor without the stiffness limit", "double taup = fmax(tau, fabs(dt));",
     "double taup = tau;"),
    ("predictor advancing a full step", "double coef = 0.5 * dt * P->sp_mass[sp] / taup;",
     "double coef = dt * P->sp_mass[sp] / taup;"),
    ("predictor drag sign", "for (int c = 0; c < 3; c++) J[c] = coef * (pn[c] - vg[c]);",
     "for (int c = 0; c < 3; c++) J[c] = coef * (vg[c] - pn[c]);"),
    ("semi-implicit orbital-advection Lambda without (1 - q/2)",
     "l10 = (1.0 - 0.5 * qq) * Om * dt;", "l10 = Om * dt;"),
    ("semi-implicit standard-frame Lambda sign", "                    l10 = Om * dt;\n",
     "                    l10 = -Om * dt;\n"),
    ("volume weighting linear in R", "if (b >= 0.0 || a <= 0.0) return fabs((a - b) * (a + b));",
     "if (b >= 0.0 || a <= 0.0) return fabs(a - b);"),
    ("volume weighting ghost centre half a zone out",
     "if (k < 0) return 0.5 * (edges[0] + edges[1]) - (edges[1] - edges[0]);",
     "if (k < 0) return 0.5 * (edges[0] + edges[1]) - 0.5 * (edges[1] - edges[0]);"),
    ("volume weighting polar shell signed across the pole",
     "total += fabs(2.0 * sin(0.5 * (u + v)) * sin(0.5 * (v - u)));",
     "total += 2.0 * sin(0.5 * (u + v)) * sin(0.5 * (v - u));"),
    ("volume weighting r^2 instead of r^3", "return (a - b) * (a * a + a * b + b * b);",
     "return (a - b) * (a + b);"),
    ("mass deposit without the z weight", "mass[idx] += m * (w[0][a] * w[1][b] * w[2][c]);",
     "mass[idx] += m * (w[0][a] * w[1][b]);"),
    ("mass deposit with species 0 for every grain",
     "double m = P->sp_mass[species ? species[g] : 0];", "double m = P->sp_mass[0];"),
    ("Epstein stopping time value times rho", "if (mode == OT_EPSTEIN) return value / rho_g;",
     "if (mode == OT_EPSTEIN) return value * rho_g;"),
    ("Epstein with the host zone's density instead of the gathered one",
     "double tau = stopping_time(P, mode, value, qm, rg);",
     "double tau = stopping_time(P, mode, value, qm, rho[node_index(host[0], 0, n0, P->bc[0])"
     " + (int64_t)n0 * (node_index(host[1], 0, n1, P->bc[1])"
     " + (int64_t)n1 * node_index(host[2], 0, n2, P->bc[2]))]);"),
    ("orbital-advection energy channel with p^n",
     "            a[2] = zf;\n            dHdp[0] = vh[0]; dHdp[1] = vh[1]; dHdp[2] = vh[2];",
     "            a[2] = zf;\n            if (P->fargo) { dHdp[0] = pn[0]; dHdp[1] = pn[1]; "
     "dHdp[2] = pn[2]; } else { dHdp[0] = vh[0]; dHdp[1] = vh[1]; dHdp[2] = vh[2]; }"),
    ("orbital-advection energy channel with the total velocity",
     "            a[2] = zf;\n            dHdp[0] = vh[0]; dHdp[1] = vh[1]; dHdp[2] = vh[2];",
     "            a[2] = zf;\n            dHdp[0] = vh[0]; dHdp[1] = vh[1] - (P->fargo ? qq * Om * qm[0]"
     " : 0.0); dHdp[2] = vh[2];"),
    ("orbital-advection non-frictional force without the shear",
     "                a[1] = (qq - 2.0) * Om * vh[0];\n            }\n            a[2] = zf;",
     "                a[1] = -2.0 * Om * vh[0];\n            }\n            a[2] = zf;"),
    ("fixed point: host rounded on its own, not the rest",
     "        fixed[4 * hidx + ch] += rest;",
     "        fixed[4 * hidx + ch] += (int64_t)llrint(w[0][1] * w[1][1] * w[2][1] * D[ch] / quantum);"),
    ("fixed point: pieces truncated instead of rounded",
     "int64_t piece = (int64_t)llrint(W * D[ch] / quantum);",
     "int64_t piece = (int64_t)(W * D[ch] / quantum);"),
]


def _run_mutant(case, workdir):
    name, orig, planted = case
    src = open(SRC).read()
    assert src.count(orig) == 1, name
    d = os.path.join(workdir, "m%d" % MUTATIONS.index(case))
    os.makedirs(d)
    c = os.path.join(d, "dust_oracle.c")
    with open(c, "w") as f:
        f.write(src.replace(orig, planted))
    lib = os.path.join(d, "liboracle.so")
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-std=c99", "-o", lib, c, "-lm"])
    env = dict(os.environ, DUST_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"]
                       + PIN_SUITES, cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    return name, r.returncode


def test_every_planted_mistake_fails_a_pin():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    work = tempfile.mkdtemp(prefix="oracle_mut_")
    try:
        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
            results = list(ex.map(lambda c: _run_mutant(c, work), MUTATIONS))
    finally:
        shutil.rmtree(work, ignore_errors=True)
    survived = [name for name, rc in results if rc == 0]
    assert not survived, "pins did not catch: %s" % survived
