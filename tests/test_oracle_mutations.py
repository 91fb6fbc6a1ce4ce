"""The oracle's pins catch plausible mistakes.

Each case plants one slip in a scratch copy of the oracle's C source (a wrong
direction index, a dropped or mis-signed term, a swapped relaxation time, a
wrong boundary population, a wrong transpose in the adjoint...), rebuilds
that copy and runs the forward or adjoint pin tests against it in a
subprocess; at least one pin must fail.  The real oracle is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = [
    ("opposite of a diagonal", "static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};",
     "static const int OPP[9] = {0, 3, 4, 1, 2, 8, 7, 6, 5};"),
    ("equilibrium 9/2 term", "4.5 * eu * eu", "4.0 * eu * eu"),
    ("equilibrium 3/2 u^2 term", "- 1.5 * uu", "- 1.0 * uu"),
    ("scalar c_s^2 fixed at 1/3", "return wg(L, i) * C * (1.0 + eu / cs2);",
     "return wg(L, i) * C * (1.0 + 3.0 * eu);"),
    ("scalar relaxes with tau_f", "(gn[i] - geq(L, i, C, ux, uy)) / L->tau_g",
     "(gn[i] - geq(L, i, C, ux, uy)) / L->tau_f"),
    ("fluid relaxation rate", "(fn[i] - feq(i, rho, ux, uy)) / L->tau_f",
     "(fn[i] - feq(i, rho, ux, uy)) * (1.0 - 0.5 / L->tau_f)"),
    ("fluid bounce-back keeps direction", "L->f[c * 9 + OPP[i]] = L->fp[c * 9 + i];",
     "L->f[c * 9 + i] = L->fp[c * 9 + i];"),
    ("scalar bounce-back keeps direction", "L->g[c * 5 + OPP[i]] = L->gp[c * 5 + i];",
     "L->g[c * 5 + i] = L->gp[c * 5 + i];"),
    ("Zou-He tangential correction sign", "fn[diag_in_up] = fn[diag_out_dn] - 0.5 * (fn[2] - fn[4])",
     "fn[diag_in_up] = fn[diag_out_dn] + 0.5 * (fn[2] - fn[4])"),
    ("Zou-He diagonal momentum sign", "fn[diag_in_dn] = fn[diag_out_up] + 0.5 * (fn[2] - fn[4]) +\n"
     "                     s * (1.0 / 6.0) * jx;",
     "fn[diag_in_dn] = fn[diag_out_up] + 0.5 * (fn[2] - fn[4]) -\n"
     "                     s * (1.0 / 6.0) * jx;"),
    ("Zou-He side sign dropped", "fn[axis_in] = fn[axis_out] + s * (2.0 / 3.0) * jx;",
     "fn[axis_in] = fn[axis_out] + (2.0 / 3.0) * jx;"),
    ("Zou-He diagonal weight", "fn[diag_out_dn] - 0.5 * (fn[2] - fn[4]) +\n                     s * (1.0 / 6.0) * jx;",
     "fn[diag_out_dn] - 0.5 * (fn[2] - fn[4]) +\n                     s * (1.0 / 3.0) * jx;"),
    ("Zou-He velocity density", "rho = K / (1.0 - s * ux);", "rho = K / (1.0 + s * ux);"),
    ("Zou-He pressure velocity sign", "ux = s * (1.0 - K / rho);", "ux = s * (K / rho - 1.0);"),
    ("held concentration on the wrong population", "int g_in = s > 0 ? 1 : 3;", "int g_in = s > 0 ? 3 : 1;"),
    ("do-nothing outlet left as a wall", "gn[g_in] = L->gp[c * 5 + g_in];", "(void)0;"),
    ("free flight against e_i",
     "int xn = x + EX[i], yn = y + EY[i];\n                if (L->periodic) {\n                    xn = (xn + nx) % nx;\n"
     "                    yn = (yn + ny) % ny;\n                }\n                if (is_fluid(L, xn, yn))\n"
     "                    L->g",
     "int xn = x - EX[i], yn = y - EY[i];\n                if (L->periodic) {\n                    xn = (xn + nx) % nx;\n"
     "                    yn = (yn + ny) % ny;\n                }\n                if (is_fluid(L, xn, yn))\n"
     "                    L->g"),
    ("y momentum from e_x", "jy += fn[i] * EY[i];", "jy += fn[i] * EX[i];"),
    ("scalar axis weight ignores w0", "return i == 0 ? L->w0 : 0.25 * (1.0 - L->w0);",
     "return i == 0 ? L->w0 : 0.25;"),
    ("valve bit inverted", "if (!((open_mask >> P->channel) & 1u)) continue;\n        int s",
     "if (((open_mask >> P->channel) & 1u)) continue;\n        int s"),
    ("outlet mass flux without u", "q += r * ux;", "q += r;"),
    ("outlet scalar flux without u", "qc += scalar_moment(L->g + (size_t)c * 5) * ux;",
     "qc += scalar_moment(L->g + (size_t)c * 5);"),
    ("flux over velocity ports too",
     "if ((P->kind != ORC_PRESSURE && P->kind != ORC_PRESSURE_RESCALE) || !((open_mask >> P->channel) & 1u))",
     "if (!((open_mask >> P->channel) & 1u))"),
    ("diagonal weight", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 18.0};"),
]

# slips in the adjoint, caught by tests/test_oracle_adjoint.py
ADJOINT_MUTANTS = [
    ("adjoint: equilibrium u^2 term", "Ar += af[k] * W9[k] * (1.0 - 4.5 * eu * eu + 1.5 * uu);",
     "Ar += af[k] * W9[k] * (1.0 - 4.5 * eu * eu);"),
    ("adjoint: momentum derivative", "Ax += af[k] * W9[k] * (3.0 * EX[k] + 9.0 * eu * EX[k] - 3.0 * ux);",
     "Ax += af[k] * W9[k] * (3.0 * EX[k] + 9.0 * eu * EX[k]);"),
    ("adjoint: scalar-to-fluid coupling dropped", "Bx += ag[k] * wk * C * EX[k] / (rho * cs2);", "(void)0;"),
    ("adjoint: relaxation-rate derivative sign", "dwg += ag[k] * (geq(L, k, C, ux, uy) - gn[k]);",
     "dwg += ag[k] * (gn[k] - geq(L, k, C, ux, uy));"),
    ("adjoint: do-nothing term lost", "pg[c * 5 + g_in] += dn[c];", "(void)dn[c];"),
    ("adjoint: Zou-He momentum weight", "double G = s * (2.0 / 3.0) * a_ax + s * (1.0 / 6.0) * (a_up + a_dn);",
     "double G = s * (2.0 / 3.0) * a_ax + s * (1.0 / 3.0) * (a_up + a_dn);"),
    ("adjoint: Zou-He velocity derivative", "du = G * K / (den * den);", "du = G * K / den;"),
    ("adjoint: Dirichlet transpose sign", "if (i != g_in) b[i] -= ain;", "if (i != g_in) b[i] += ain;"),
    ("adjoint: bounce-back transpose keeps direction", "else pf[c * 9 + i] = bf[c * 9 + OPP[i]];",
     "else pf[c * 9 + i] = bf[c * 9 + i];"),
]


# slips in the decay term and the paper's rescaling ports, caught by
# tests/test_oracle_paper_bc.py
PAPER_BC_MUTANTS = [
    ("decay adds compound", "double R = -L->decay * C;  /* reaction term of Eq. cde */",
     "double R = L->decay * C;  /* reaction term of Eq. cde */"),
    ("decay on every population", "+ wg(L, i) * R;\n        }\n}", "+ R;\n        }\n}"),
    ("decay skipped in the scalar-only step",
     "L->gp[c * 5 + i] = gn[i] - (gn[i] - geq(L, i, C, ux[c], uy[c])) / L->tau_g + wg(L, i) * R;",
     "L->gp[c * 5 + i] = gn[i] - (gn[i] - geq(L, i, C, ux[c], uy[c])) / L->tau_g;"),
    ("rescale factor inverted", "double gamma = rho_port / sum;", "double gamma = sum / rho_port;"),
    ("port unknowns not carried over", "for (int k = 0; k < 3; ++k) fn[unknown[k]] = fpn[unknown[k]];",
     "(void)fpn;"),
    ("port unknowns of the other side", "int unknown[3] = {s > 0 ? 1 : 3, s > 0 ? 5 : 6, s > 0 ? 8 : 7};",
     "int unknown[3] = {s > 0 ? 3 : 1, s > 0 ? 7 : 8, s > 0 ? 6 : 5};"),
    ("scalar rescaled to 1", "double gamma = C_in / sum;", "double gamma = 1.0 / sum;"),
    ("scalar fallback at rest", "for (int i = 0; i < 5; ++i) gn[i] = geq(L, i, C_in, ux, uy);",
     "for (int i = 0; i < 5; ++i) gn[i] = geq(L, i, C_in, 0.0, 0.0);"),
    ("wall momentum halved instead of a third", "jx = m1[1] / 3.0;\n        jy = m1[2] / 3.0;",
     "jx = m1[1] / 2.0;\n        jy = m1[2] / 2.0;"),
    ("wall density not extrapolated", "rho = is_fluid(L, x2, y2) ? 2.0 * m1[0] - M[(size_t)node(L, x2, y2) * 3] : m1[0];",
     "rho = m1[0];"),
    ("wall neighbours behind the node", "int x1 = x + EX[m], y1 = y + EY[m], x2 = x + 2 * EX[m], y2 = y + 2 * EY[m];",
     "int x1 = x - EX[m], y1 = y - EY[m], x2 = x - 2 * EX[m], y2 = y - 2 * EY[m];"),
]

CASES = [m + ("tests/test_oracle_pins.py",) for m in MUTANTS] + \
        [m + ("tests/test_oracle_adjoint.py",) for m in ADJOINT_MUTANTS] + \
        [m + ("tests/test_oracle_paper_bc.py",) for m in PAPER_BC_MUTANTS]


@pytest.mark.parametrize("name,old,new,pins", CASES, ids=[m[0] for m in CASES])
def test_a_planted_mistake_fails_a_pin(tmp_path, name, old, new, pins):
    src = open(os.path.join(ROOT, "oracle", "lbm_oracle.c")).read()
    assert src.count(old) >= 1, "mutation site not found: " + name
    for sub in ("oracle", "tests"):
        shutil.copytree(os.path.join(ROOT, sub), tmp_path / sub,
                        ignore=shutil.ignore_patterns("*.so", "__pycache__", "golden"))
    pkg = tmp_path / "paper_1307_4703_gb300"
    pkg.mkdir()
    for f in ("__init__.py", "workloads.py"):
        shutil.copy(os.path.join(ROOT, "paper_1307_4703_gb300", f), pkg / f)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")
    (tmp_path / "oracle" / "lbm_oracle.c").write_text(src.replace(old, new, 1))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", pins],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "no pin caught the planted mistake '%s'" % name
    assert "failed" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
