"""Plant plausible mistakes in a copy of the oracle and check that the pins catch them.

Each mutant is a one-line edit of ``oracle/band_oracle.c`` (a dropped term, a wrong
index, a flipped sign, a transposed operand), compiled into a temporary library and
loaded by the pin tests through BAND_ORACLE_LIB.  The pins must fail for every one.
Runs on the CPU only.

Edits that no pin can see because they change nothing the oracle returns are not
listed: computing the product P = M X of the Hotelling-Bodewig step on w + 1 rather
than w + 2 diagonals (the update X (2I - P) reads only w of them); reading the stored
X through one diagonal fewer than it keeps (an off-by-one in band_get's offset test: for
triangular M the outermost diagonal of X (2I - M X) is rebuilt exactly from the inner
ones once those are exact, which is no later than the correct iteration gets there, so
every iterate comes out the same); and keeping the negative powers of x_i(t) in the
symbolic back-substitution (after the residue flush they are zero).
"""
import concurrent.futures
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "band_oracle.c")

MUTANTS = {
    "npdm_gamma_wrong_index": ("g = op_sub(b[i], op_mul(alpha[i - 2], a[i], ops), ops);",
                               "g = op_sub(b[i], op_mul(alpha[i - 1], a[i], ops), ops);"),
    "npdm_mu_dropped_beta": ("if (i >= 2) m = op_sub(m, op_mul(beta[i - 2], a[i], ops), ops);", ""),
    "npdm_back_sign": ("x[i] = op_sub(xi, op_mul(beta[i], x[i + 2], ops), ops);",
                       "x[i] = op_add(xi, op_mul(beta[i], x[i + 2], ops), ops);"),
    "npdm_z_dropped_term": ("if (i >= 2) zi = op_sub(zi, op_mul(z[i - 2], a[i], ops), ops);", ""),
    "ntdm_transposed_operand": ("if (i <= n - 2) alpha[i] = op_div(d[i], mu, ops);",
                                "if (i <= n - 2) alpha[i] = op_div(b[i + 1], mu, ops);"),
    "gepp_rhs_not_swapped": ("double t = x[j]; x[j] = x[p]; x[p] = t;", ""),
    "laurent_division_sign": ("s = dd_add(s, dd_neg(p));", "s = dd_add(s, p);"),
    "dd_residue_not_flushed": ("if (fabs(v.hi) <= DD_RESIDUE * mag) return dd_of(0.0);", ""),
    "dd_product_error_dropped": ("double e = fma(x.hi, y.hi, -p);", "double e = 0.0;"),
    "dd_two_sum_error_dropped": ("dd r = {s, (a - av) + (b - bv)};", "dd r = {s, 0.0};"),
    "dd_div_one_digit": ("return dd_add(quick_two_sum(q1, q2), dd_of(q3));", "return dd_of(q1);"),
    "symbolic_det_wrong_factor": ("det_push(&D, 0, fac[n + i]);", "det_push(&D, 0, fac[i]);"),
    "symbolic_td_reads_a": ("const double* pa = k == 2 ? a : zero;", "const double* pa = a;"),
    "symbolic_window_short": ("#define LP 16", "#define LP 3"),
    "ilu0_wrong_operand": ("w[2] = w[2] - w[0] * u2[i - 2];", "w[2] = w[2] - w[0] * u1[i - 2];"),
    "hb_missing_2I": ("double y = (m == j ? 2.0 : 0.0) - band_get(P, n, wp, lower, m, j);",
                      "double y = (m == j ? 1.0 : 0.0) - band_get(P, n, wp, lower, m, j);"),
    "sip_residual_sign": ("r[i] = op_sub(f[i], s, ops);", "r[i] = op_sub(s, f[i], ops);"),
    "refine_missing_rescale": ("double dl = s * (double)x32[i];", "double dl = (double)x32[i];"),
    "adjoint_not_transposed": ("if (i >= 1) tb[i] = d[i - 1];", "if (i >= 1) tb[i] = b[i];"),
    "lu_minus_a_sign": ("ka[i] = i >= 2 ? lu_a - a[i] : 0.0;", "ka[i] = i >= 2 ? a[i] - lu_a : 0.0;"),
    "refine_absolute_stop": ("if (dmax <= rel_stop * xmax) break;", "if (dmax <= rel_stop) break;"),
    "ntdm_back_sign": ("x[i] = op_sub(z[i], op_mul(alpha[i], x[i + 1], ops), ops);",
                       "x[i] = op_add(z[i], op_mul(alpha[i], x[i + 1], ops), ops);"),
    "hb_start_not_inverse": ("X[i] = 1.0 / dg;", "X[i] = dg;"),
    "hb_band_wrong_side": ("int64_t off = lower ? i - j : j - i;\n  if (off < 0 || off >= w) return 0.0;",
                           "int64_t off = lower ? j - i : i - j;\n  if (off < 0 || off >= w) return 0.0;"),
    "hb_update_one_diagonal_short": ("for (int mo = 0; mo < w; ++mo) {",
                                     "for (int mo = 0; mo < w - 1; ++mo) {"),
    "mnpdm_e_elim_drops_b": ("if (i >= 1) B[i] = op_sub(B[i], op_mul(m, i + 1 >= 2 ? a[i + 1] : 0.0, ops), ops);",
                             ""),
    "mnpdm_a_elim_wrong_row": ("C[i] = op_sub(C[i], op_mul(m, D[i - 1], ops), ops);",
                               "C[i] = op_sub(C[i], op_mul(m, C[i - 1], ops), ops);"),
    "mnpdm_rhs_not_eliminated": ("F[i] = op_sub(F[i], op_mul(m, F[i + 1], ops), ops);", ""),
    "sip2d_fill_dropped_from_k": ("if (in_grid(nx, ny, k, 1, -1)) v += ls[k] * AE(k - nx) * x[k - nx + 1];",
                                  ""),
    "sip2d_fill_wrong_column": ("if (in_grid(nx, ny, k, -1, 1)) v += lw[k] * AT(k - 1) * x[k + nx - 1];",
                                "if (in_grid(nx, ny, k, -1, 1)) v += lw[k] * AT(k - 1) * x[k + nx];"),
    "ilu0_2d_wrong_u_entry": ("      v -= ls[k] * t[k - nx];", "      v -= ls[k] * e[k - nx];"),
    "symbolic_residue_pivot_ignored": ("if (st == ORC_OK && residue_pivot(n, pa, b, c, fac)) st = ORC_ZERO_PIVOT;",
                                       ""),
    "cond1_not_transposed": ("if (orc_gepp_band(n, k, ta, tb, tc, td, te, y, z, NULL) != ORC_OK)",
                             "if (orc_gepp_band(n, k, a, b, c, d, e, y, z, NULL) != ORC_OK)"),
    "batch_strides_swapped": ("int64_t p = off + i * J->elem_stride;", "int64_t p = off + i * J->sys_stride;"),
    "batch_bandwidths_ignored": ("int k = J->hbw ? J->hbw[s] : J->k;", "int k = J->k;"),
}


def _run_mutant(name, workdir):
    """Compile the oracle with one planted mistake and run the pins against it;
    returns (pins' exit code, the end of their output)."""
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor must be unique: " + name
    mutated = os.path.join(workdir, name + ".c")
    with open(mutated, "w") as fh:
        fh.write(src.replace(old, new))
    lib = os.path.join(workdir, "lib" + name + ".so")
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared", "-pthread",
                    "-o", lib, mutated, "-lm"], check=True)
    env = dict(os.environ, BAND_ORACLE_LIB=lib)
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return res.returncode, res.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Every mutant's pin run, several at a time (each run is its own process)."""
    workdir = str(tmp_path_factory.mktemp("mutants"))
    workers = max(1, min(8, os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(workers) as pool:
        futures = {name: pool.submit(_run_mutant, name, workdir) for name in MUTANTS}
        return {name: fut.result() for name, fut in futures.items()}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, outcomes):
    code, tail = outcomes[name]
    assert code != 0, "pins did not catch mutant %s:\n%s" % (name, tail)
