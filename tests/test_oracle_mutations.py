"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle/ccell_oracle.c`` (on the
CPU, in a temporary directory), builds it, and runs the pin suite against that
build; the suite has to fail.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ccell_oracle.c")

MUTATIONS = {
    "wrong face radius in A (r_e for r_w)":
        ("const double A = -r_w * lw", "const double A = -r_e * lw"),
    "sign of the south flux in Lambda_j":
        ("const double Lj = (fn - fs) / etabar;", "const double Lj = (fn + fs) / etabar;"),
    "north face conductivity from the south neighbour":
        ("? lam_face(p, m, T0, Tn[i]) * (Tn[i] - T0) / eta_n", "? lam_face(p, m, T0, Ts[i]) * (Tn[i] - T0) / eta_n"),
    "face conductivity at one node instead of the face mean":
        ("return lam_m(p, m, 0.5 * (Ta + Tb));", "return lam_m(p, m, Ta);"),
    "heat capacity saturation squared instead of cubed":
        ("(1.0 + y * y * y)", "(1.0 + y * y)"),
    "density dropped from rho c":
        ("const double rc = p->rho[m] * cap_m(p, m, T0);\n    /* Eq. (Lambda_j)",
         "const double rc = cap_m(p, m, T0);\n    /* Eq. (Lambda_j)"),
    "interface row with the cell widths swapped":
        ("a[i] = -lm * h_e;\n      c[i] = -lp * h_w;\n      b[i] = lm * h_e + lp * h_w;",
         "a[i] = -lm * h_w;\n      c[i] = -lp * h_e;\n      b[i] = lm * h_w + lp * h_e;"),
    "interface recursion with the cell widths swapped":
        ("const double lmh = -ra[i], lph = -rcv[i];", "const double lmh = -rcv[i], lph = -ra[i];"),
    "source term dropped from F":
        ("F = rc / tau * T0 + Lj + X;", "F = rc / tau * T0 + Lj;"),
    "Neumann closure at r_max dropped":
        ("beta[Nj - 1] / (1.0 - alpha[Nj - 1])", "beta[Nj - 1]"),
    "sign of alpha in the forward sweep":
        ("alpha[i] = -rcv[i] / den;", "alpha[i] = rcv[i] / den;"),
    "stability bound with eta instead of eta^2":
        ("if (e * e < eta2) eta2 = e * e;", "if (e < eta2) eta2 = e;"),
    "rectangle pulse closed interval":
        ("return (phi < p->t_on) ? 1.0 : 0.0;", "return (phi <= p->t_on) ? 1.0 : 0.0;"),
    "Dirichlet row at z = 0 copied from line 1":
        ("Th[i] = p->bc_z0 ? p->t_dirichlet : Th[(size_t)nr + i];", "Th[i] = Th[(size_t)nr + i];"),
    "sign of the heat through a Dirichlet z = 0 face":
        ("(Ts[i] - Tj[i]) / eta_s;", "(Tj[i] - Ts[i]) / eta_s;"),
    "Dirichlet value at r_max dropped":
        ("beta[Nj - 1] / (1.0 - alpha[Nj - 1]) : p->t_dirichlet;", "beta[Nj - 1] / (1.0 - alpha[Nj - 1]) : 0.0;"),
    "conductivity scale dropped":
        ("b[4] * T * T * T * T;\n    }\n  }\n  return p->lam_scale[m] * v;",
         "b[4] * T * T * T * T;\n    }\n  }\n  return v;"),
    "polynomial heat capacity read in reverse order":
        ("v = a[0] + a[1] * T + a[2] * T * T + a[3] * T * T * T;",
         "v = a[3] + a[2] * T + a[1] * T * T + a[0] * T * T * T;"),
    "resistivity 1/T instead of 1/sqrt(T)":
        ("double g = (p->g_model == 1) ? p->g_ref / sqrt(T) : 1.0;",
         "double g = (p->g_model == 1) ? p->g_ref / T : 1.0;"),
    "minimum of one cell per layer instead of two":
        ("if (n[m] < 2) n[m] = 2;", "if (n[m] < 1) n[m] = 1;"),
    "ADI: sign of the Dirichlet z = 0 value folded into the first row":
        ("if (p->bc_z0) { f[1] -= a[1] * p->t_dirichlet; }", "if (p->bc_z0) { f[1] += a[1] * p->t_dirichlet; }"),
    "ADI: Dirichlet r_max column taken as Neumann":
        ("Hj[N] = p->bc_rmax ? p->t_dirichlet : Hj[N - 1];", "Hj[N] = Hj[N - 1];"),
    "stored heat with the capacity at That":
        ("kadd(&e[0], &c[0], V * p->rho[m] * cap_m(p, m, Tj[i]) * (Hj[i] - Tj[i]));",
         "kadd(&e[0], &c[0], V * p->rho[m] * cap_m(p, m, Hj[i]) * (Hj[i] - Tj[i]));"),
    "heat through the z = 0 face always booked as Dirichlet":
        ("int k = p->bc_z0 ? 2 : 4;", "int k = 2;"),
    "rectangle pulses before t_start":
        ("  if (p->waveform == 0) {\n    if (u < 0.0) return 0.0;",
         "  if (p->waveform == 0) {\n    if (u < -1.0) return 0.0;"),
    "tanh edges of the current period only":
        ("  double k = floor((u - 0.5 * p->t_on) / p->t_period + 0.5);\n  if (k < 0.0) k = 0.0;\n"
         "  double phi = u - k * p->t_period;\n  return 0.5",
         "  double k = floor(u / p->t_period);\n  if (k < 0.0) k = 0.0;\n"
         "  double phi = u - k * p->t_period;\n  return 0.5"),
    "trace surface value from line 1":
        ("      trace[2 * n] = T[N];\n      trace[2 * n + 1] = acc / wsum;\n    }\n  }\n  if (energy)",
         "      trace[2 * n] = T[(size_t)nr + N];\n      trace[2 * n + 1] = acc / wsum;\n    }\n  }\n  if (energy)"),
    "outline with line 1 narrow accepted":
        ("if (*j_narrow < 2) return -1;", "if (*j_narrow < 1) return -1;"),
    "outline ends one node beyond the interface":
        ("if (rclass[i] == OR_IFACE && ++k == p->step_layers) { *i_step = i; break; }",
         "if (rclass[i] == OR_IFACE && ++k == p->step_layers) { *i_step = i + 1; break; }"),
    "half-cell placement: Dirichlet r_max node off the boundary":
        ("double off_hi = p->bc_rmax ? 0.0 : 0.5;", "double off_hi = 0.5;"),
    "adjoint: loss seed without the factor 2":
        ("lam[(size_t)j * nr + N] += 2.0 * tau * e * w[j];", "lam[(size_t)j * nr + N] += tau * e * w[j];"),
    "transient sub-step tau* = tau":
        ("return 1.0 - exp(-phi / (7.0 * (p->edge_w / 100.0)));", "return 1.0 - exp(-phi / (7.0 * p->edge_w));"),
    # discrete adjoint
    "adjoint: lambda term of the north flux derivative dropped":
        ("d0 += (ln_a * dN - ln) / eta_n / etabar", "d0 += (ln_a * dN) / eta_n / etabar"),
    "adjoint: south-neighbour derivative with the wrong sign":
        ("xbs[i] += X * (-ls_a * dS + ls) / eta_s / etabar;", "xbs[i] += X * (ls_a * dS + ls) / eta_s / etabar;"),
    "adjoint: heat-capacity derivative without the saturation term":
        ("v = p->c0[m] * (3.0 * x * x / p->t_ref[m] / d - x * x * x * 3.0 * y * y / p->theta[m] / (d * d));",
         "v = p->c0[m] * (3.0 * x * x / p->t_ref[m] / d);"),
    "adjoint: untransposed line solve":
        ("const double sub = c[i - 1], sup = (i < N) ? a[i + 1] : 0.0;",
         "const double sub = a[i], sup = (i < N) ? c[i] : 0.0;"),
    "adjoint: pulse-duration derivative with the wrong sign":
        ("return 0.5 * (1.0 - th * th) / p->edge_w;", "return -0.5 * (1.0 - th * th) / p->edge_w;"),
    "adjoint: Neumann row z=0 not folded into line 1":
        ("if (!p->bc_z0) mu[(size_t)nr + i] += mu[i];", "(void)0;"),
    # stepped outline
    "outline: axial face to an outside node left open":
        ("(wide_n || i <= i_step)", "(1)"),
    "outline: narrow lines solved over the full width":
        ("const int Nj = (j >= j_narrow) ? i_step : N;\n        line_rows(",
         "const int Nj = N;\n        line_rows("),
    "outline: trace over every line":
        ("for (int j = 0; j <= M && j < j_narrow; j++) {", "for (int j = 0; j <= M; j++) {"),
    "outline: Dirichlet row reset beyond the step":
        ("Th[(size_t)M * nr + i] = (i > NM) ?", "Th[(size_t)M * nr + i] = (i > N) ?"),
    "outline: narrow line's outer edge booked as an interface edge":
        ("const int ce = (i + 1 == Nj) ? OR_OUTER : cls[i + 1];", "const int ce = cls[i + 1];"),
    "outline: heat booked through the closed face at z_max":
        ("if (j == M - 1 && i <= NM) {", "if (j == M - 1) {"),
    "adjoint: Neumann row z = z_max not folded into line M-1":
        ("if (!p->bc_zmax) mu[(size_t)(M - 1) * nr + i] += mu[(size_t)M * nr + i];", "(void)0;"),
    "adjoint: cap_scale partial with the wrong sign":
        ("gbar[2 + L + m] += X * rc / tau * (T0 - yj[i]) / p->cap_scale[m];",
         "gbar[2 + L + m] += X * rc / tau * (yj[i] - T0) / p->cap_scale[m];"),
    "adjoint: derivative of the resistivity dropped":
        ("if (m == p->src_layer) d0 += p->q0 * s * src_dg(p, T0);", "(void)0;"),
    # ADI variant
    "ADI: radial term of the second half step partly at T^n":
        ("const double Li = (r_e * le * (Sj[i + 1] - Sj[i]) / h_e -",
         "const double Li = (r_e * le * (Tj[i + 1] - Tj[i]) / h_e -"),
    "ADI: full time step in the second half step's diagonal":
        ("b[j] = rc / h - a[j] - c[j];", "b[j] = rc / tau - a[j] - c[j];"),
    "ADI: source dropped from the second half step":
        ("f[j] = rc / h * Sj[i] + Li + source(p, m, T0, s);", "f[j] = rc / h * Sj[i] + Li;"),
    "ADI: Neumann closure at z = 0 not folded":
        ("} else { b[1] += a[1]; }", "} else { (void)0; }"),
    "ADI: interface cell widths swapped":
        ("Hj[i] = (lm * h_e * Hj[i - 1] + lp * h_w * Hj[i + 1])",
         "Hj[i] = (lm * h_w * Hj[i - 1] + lp * h_e * Hj[i + 1])"),
}


PIN_FILES = ["test_oracle_outline.py", "test_oracle_adi.py", "test_oracle_pins.py",
             "test_oracle_adjoint.py", "test_paper_model.py"]


CONTROL = "(no mutation)"


def _run_mutant(name, workdir):
    """Build one mutant (or the unchanged oracle for CONTROL) and run the pin
    suite against it; returns (returncode, output)."""
    old, new = MUTATIONS.get(name, ("", ""))
    src = open(SRC).read()
    if name != CONTROL and src.count(old) != 1:
        return None, f"mutation anchor not found once: {old!r}"
    d = os.path.join(workdir, str(len(name)) + "_" + str(abs(hash(name))))
    os.makedirs(d)
    mut, so = os.path.join(d, "mutant.c"), os.path.join(d, "libmutant.so")
    with open(mut, "w") as f:
        f.write(src.replace(old, new) if name != CONTROL else src)
    cc = shutil.which("gcc") or shutil.which("cc")
    subprocess.run([cc, "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", mut,
                    "-o", so, "-lm"], check=True, capture_output=True)
    # one thread per mutant: the mutants run side by side
    env = dict(os.environ, CCELL_ORACLE_SO=so, OMP_NUM_THREADS="1")
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"]
                         + [os.path.join(ROOT, "tests", f) for f in PIN_FILES],
                         env=env, capture_output=True, text=True, cwd=ROOT)
    return res.returncode, res.stdout[-2000:]


@pytest.fixture(scope="module")
def mutant_results(tmp_path_factory):
    workdir = str(tmp_path_factory.mktemp("mutants"))
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        futures = {name: ex.submit(_run_mutant, name, workdir)
                   for name in list(MUTATIONS) + [CONTROL]}
        return {name: fut.result() for name, fut in futures.items()}


def test_unchanged_oracle_passes_the_same_runner(mutant_results):
    rc, out = mutant_results[CONTROL]
    assert rc == 0, f"the pin suite fails on the unchanged oracle in this runner:\n{out}"


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, mutant_results):
    rc, out = mutant_results[name]
    assert rc is not None, out
    assert rc != 0, f"pins did not catch: {name}\n{out}"
