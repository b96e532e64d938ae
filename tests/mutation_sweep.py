"""Mutation sweep of the oracle's pins (run by hand; not collected by pytest).

Each entry plants one plausible mistake in a scratch copy of
oracle/hji_oracle.c (a dropped term, a wrong sign, index, coefficient or
stencil, a transposed operand, a wrong stage or projection order, a changed
stopping or tie rule), rebuilds that copy and runs the CPU pins against it.
Every mutation must make at least one pin fail; a survivor is a missing pin.
The repository's own oracle is never modified.

    python tests/mutation_sweep.py [--workdir DIR] [--jobs 4] [name ...]

Prints one line per mutation (KILLED with the first failing test, or
SURVIVED) and exits 1 if any survived or a pattern no longer matches the
oracle's source exactly once.
"""
import argparse
import os
import shutil
import subprocess
import sys
import tempfile
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_TESTS = ["tests/test_oracle_definitions.py", "tests/test_oracle_solver.py",
             "tests/test_oracle_operators.py", "tests/test_oracle_control.py",
             "tests/test_oracle_discount.py", "tests/test_workloads.py"]

# (name, text in oracle/hji_oracle.c, replacement)
MUTATIONS = [
    ('spacing_periodic',
     'if (P->periodic[a]) return (P->hi[a] - P->lo[a]) / (double)P->n[a];',
     'if (P->periodic[a]) return (P->hi[a] - P->lo[a]) / (double)(P->n[a] - 1);'),
    ('spacing_nonperiodic',
     'return (P->hi[a] - P->lo[a]) / (double)(P->n[a] - 1);\n}',
     'return (P->hi[a] - P->lo[a]) / (double)(P->n[a]);\n}'),
    ('ghost_constant',
     'return edge + k * (edge - inner);',
     'return edge;'),
    ('ghost_k_dropped',
     'return edge + k * (edge - inner);',
     'return edge + (edge - inner);'),
    ('ghost_sign',
     'return edge + k * (edge - inner);',
     'return edge - k * (edge - inner);'),
    ('ghost_low_inner',
     'j[a] = 1;\n        inner',
     'j[a] = 2;\n        inner'),
    ('ghost_high_inner',
     'j[a] = N - 2;',
     'j[a] = N - 3;'),
    ('periodic_as_extrap',
     'if (P->periodic[a]) {\n        int64_t w',
     'if (0) {\n        int64_t w'),
    ('dyn_A_sign',
     'fi += P->A[i * OR_MAXD + j] * x[j];',
     'fi -= P->A[i * OR_MAXD + j] * x[j];'),
    ('dyn_A_transposed',
     'fi += P->A[i * OR_MAXD + j] * x[j];',
     'fi += P->A[j * OR_MAXD + i] * x[j];'),
    ('dyn_terms_dropped',
     'fi += P->term_w[t] * apply_fn',
     'fi += 0.0 * P->term_w[t] * apply_fn'),
    ('fn_tan_sin',
     'return tan(x);',
     'return sin(x);'),
    ('fn_cos_sin',
     'return cos(x);\n}',
     'return sin(x);\n}'),
    ('dyn_G_transposed',
     'fi += P->G[i * OR_MAXU + j] * u[j];',
     'fi += P->G[j * OR_MAXU + i] * u[j];'),
    ('dyn_E_sign',
     'fi += P->E[i * OR_MAXU + k] * d[k];',
     'fi -= P->E[i * OR_MAXU + k] * d[k];'),
    ('dyn_E_transposed',
     'fi += P->E[i * OR_MAXU + k] * d[k];',
     'fi += P->E[k * OR_MAXU + i] * d[k];'),
    ('dyn_const_dropped',
     'double fi = P->c[i];',
     'double fi = 0.0;'),
    ('ham_min_over_u',
     '        if (worst > best) best = worst;\n    }\n    return best;',
     '        if (best == -INFINITY || worst < best) best = worst;\n    }\n    return best;'),
    ('ham_max_over_d',
     '            if (v < worst) worst = v;\n        }\n        if (worst > best) best = worst;',
     '            if (worst == INFINITY || v > worst) worst = v;\n        }\n        if (worst > best) best = worst;'),
    ('ham_dot_short',
     '            double v = dot(P->ndim, p, f);\n            if (v < worst) worst = v;\n        }\n        if (worst > best) best = worst;',
     '            double v = dot(P->ndim - 1, p, f);\n            if (v < worst) worst = v;\n        }\n        if (worst > best) best = worst;'),
    ('alpha_no_abs',
     'if (fabs(f[a]) > alpha[a]) alpha[a] = fabs(f[a]);',
     'if (f[a] > alpha[a]) alpha[a] = f[a];'),
    ('alpha_dt_max_not_sum',
     'r += al[a] / dx[a];',
     'r = fmax(r, al[a] / dx[a]);'),
    ('alpha_dt_times_dx',
     'r += al[a] / dx[a];',
     'r += al[a] * dx[a];'),
    ('alpha_last_node',
     'if (al[a] > alpha[a]) alpha[a] = al[a];',
     'alpha[a] = al[a];'),
    ('dt_half',
     '*dt = cfl / rate;',
     '*dt = 0.5 * cfl / rate;'),
    ('eno1_pm_forward',
     '*pm = (v[c] - v[c - 1]) / dx;',
     '*pm = (v[c + 1] - v[c]) / dx;'),
    ('eno2_factor',
     '*pm = D[c - 1] / dx + smaller_magnitude(Sm, S0) / (2.0 * dx);',
     '*pm = D[c - 1] / dx + smaller_magnitude(Sm, S0) / dx;'),
    ('eno2_pp_sign',
     '*pp = D[c] / dx - smaller_magnitude(S0, Sp) / (2.0 * dx);',
     '*pp = D[c] / dx + smaller_magnitude(S0, Sp) / (2.0 * dx);'),
    ('eno2_larger',
     'return fabs(a) <= fabs(b) ? a : b;',
     'return fabs(a) >= fabs(b) ? a : b;'),
    ('eno2_Sm_index',
     'double Sm = D[c - 1] - D[c - 2];',
     'double Sm = D[c] - D[c - 2];'),
    ('eno2_pp_uses_Sm',
     '*pp = D[c] / dx - smaller_magnitude(S0, Sp)',
     '*pp = D[c] / dx - smaller_magnitude(Sm, S0)'),
    ('weno_ideal_swapped',
     'double a1 = 0.1 /',
     'double a1 = 0.3 /'),
    ('weno_ideal_swapped3',
     'double a3 = 0.3 /',
     'double a3 = 0.1 /'),
    ('weno_phi1_coef',
     'double phi1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0;',
     'double phi1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0 + 0.01 * (v1 - v3);'),
    ('weno_s2_index',
     '0.25 * (v2 - v4) * (v2 - v4);',
     '0.25 * (v2 - v3) * (v2 - v3);'),
    ('weno_s1_coef',
     '0.25 * (v1 - 4.0 * v2 + 3.0 * v3) * (v1 - 4.0 * v2 + 3.0 * v3);',
     '0.25 * (v1 - 3.0 * v2 + 2.0 * v3) * (v1 - 3.0 * v2 + 2.0 * v3);'),
    ('weno_s3_1312',
     'double s3 = 13.0 / 12.0 *',
     'double s3 = 1.0 *'),
    ('weno_no_square',
     'double a2 = 0.6 / ((s2 + eps) * (s2 + eps));',
     'double a2 = 0.6 / (s2 + eps);'),
    ('weno_eps_big',
     'double eps = 1e-6 * vmax + 1e-99;',
     'double eps = 1e-2 * vmax + 1e-99;'),
    ('weno_pp_reversed',
     '*pp = weno5(D[c + 2] / dx, D[c + 1] / dx, D[c] / dx, D[c - 1] / dx, D[c - 2] / dx);',
     '*pp = weno5(D[c - 2] / dx, D[c - 1] / dx, D[c] / dx, D[c + 1] / dx, D[c + 2] / dx);'),
    ('weno_pm_shift',
     '*pm = weno5(D[c - 3] / dx, D[c - 2] / dx, D[c - 1] / dx, D[c] / dx, D[c + 1] / dx);',
     '*pm = weno5(D[c - 2] / dx, D[c - 1] / dx, D[c] / dx, D[c + 1] / dx, D[c + 2] / dx);'),
    ('lf_pbar_forward',
     'pbar[a] = 0.5 * (pp[a] + pm[a]);',
     'pbar[a] = pp[a];'),
    ('lf_diss_sign',
     'diss += al[a] * 0.5 * (pp[a] - pm[a]);',
     'diss -= al[a] * 0.5 * (pp[a] - pm[a]);'),
    ('lf_diss_double',
     'diss += al[a] * 0.5 * (pp[a] - pm[a]);',
     'diss += al[a] * (pp[a] - pm[a]);'),
    ('lf_local_flag_inverted',
     'if (flags & OR_LOCAL_LF) oracle_alpha_point',
     'if (!(flags & OR_LOCAL_LF)) oracle_alpha_point'),
    ('rk2_wrong_stage',
     'Vout[c] = 0.5 * V[c] + 0.5 * (W1[c] + dt * L[c]);',
     'Vout[c] = 0.5 * V[c] + 0.5 * (V[c] + dt * L[c]);'),
    ('rk3_weights',
     'W2[c] = 0.75 * V[c] + 0.25 * (W1[c] + dt * L[c]);',
     'W2[c] = 0.25 * V[c] + 0.75 * (W1[c] + dt * L[c]);'),
    ('rk3_final_stage',
     'Vout[c] = V[c] / 3.0 + 2.0 * (W2[c] + dt * L[c]) / 3.0;',
     'Vout[c] = V[c] / 3.0 + 2.0 * (W1[c] + dt * L[c]) / 3.0;'),
    ('proj_max',
     'if (!(flags & OR_BRS) && l[c] < Vout[c]) Vout[c] = l[c];',
     'if (!(flags & OR_BRS) && l[c] > Vout[c]) Vout[c] = l[c];'),
    ('proj_before_discount',
     '        if (discounted) Vout[c] = gamma * Vout[c];\n        if (!(flags & OR_BRS) && l[c] < Vout[c]) Vout[c] = l[c];',
     '        if (!(flags & OR_BRS) && l[c] < Vout[c]) Vout[c] = l[c];\n        if (discounted) Vout[c] = gamma * Vout[c];'),
    ('discount_on_old',
     'if (discounted) Vout[c] = gamma * Vout[c];',
     'if (discounted) Vout[c] = Vout[c] - (1.0 - gamma) * V[c];'),
    ('delta_vs_l',
     'double ch = fabs(Vout[c] - V[c]);',
     'double ch = fabs(Vout[c] - l[c]);'),
    ('init_no_min',
     'V[c] = (k && k[c] < l[c]) ? k[c] : l[c];',
     'V[c] = k ? k[c] : l[c];'),
    ('init_max',
     'V[c] = (k && k[c] < l[c]) ? k[c] : l[c];',
     'V[c] = (k && k[c] > l[c]) ? k[c] : l[c];'),
    ('stop_rate_unscaled',
     'if (delta < tol + tol_rate * dt) {',
     'if (delta < tol + tol_rate) {'),
    ('interval_K_plus1',
     'K = (int64_t)llround(interval / dt);',
     'K = (int64_t)llround(interval / dt) + 1;'),
    ('interval_no_snap_update',
     '            memcpy(snap, V, sizeof(double) * (size_t)total);\n            if (change < interval_tol)',
     '            if (change < interval_tol)'),
    ('brs_init_min',
     'if ((flags & OR_BRS) && k) memcpy(V, k, sizeof(double) * (size_t)total);',
     'if (0) memcpy(V, k, sizeof(double) * (size_t)total);'),
    ('ctrl_tie_ge',
     '        if (worst > best) {\n            best = worst;\n            best_ub = ub;',
     '        if (worst >= best) {\n            best = worst;\n            best_ub = ub;'),
    ('ctrl_d_not_kept',
     '            best_db = worst_db;\n',
     ''),
    ('ctrl_grad_forward',
     '            pbar[a] = 0.5 * (pp + pm);\n        }\n        oracle_control_at',
     '            pbar[a] = pp;\n        }\n        oracle_control_at'),
    ('unravel_fortran',
     'for (int a = P->ndim - 1; a >= 0; --a) {\n        idx[a] = flat % P->n[a];',
     'for (int a = 0; a < P->ndim; ++a) {\n        idx[a] = flat % P->n[a];'),
    ('grad_pm_only',
     'grad[(int64_t)a * total + cidx] = 0.5 * (pp + pm);',
     'grad[(int64_t)a * total + cidx] = pm;'),
    ('periodic_wrap_off',
     'int64_t w = s % N;',
     'int64_t w = (s + 1) % N;'),
    ('weno_s2_1312',
     'double s2 = 13.0 / 12.0 *',
     'double s2 = 1.0 *'),
    ('weno_quarter',
     '0.25 * (v2 - v4) * (v2 - v4);',
     '0.5 * (v2 - v4) * (v2 - v4);'),
]


def _tree(workdir, w):
    t = os.path.join(workdir, "tree%d" % w)
    if os.path.exists(t):
        shutil.rmtree(t)
    os.makedirs(t)
    for d in ("oracle", "tests", "workloads"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(t, d),
                        ignore=shutil.ignore_patterns("__pycache__", "*.so", "*.tmp*"))
    return t


def _run_one(tree, src, mutation):
    name, old, new = mutation
    n = src.count(old)
    if n != 1:
        return name, "PATTERN MATCHES %d TIMES" % n, 0.0
    with open(os.path.join(tree, "oracle", "hji_oracle.c"), "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(tree, "oracle", "_hji_oracle.so")
    if os.path.exists(lib):
        os.remove(lib)
    env = dict(os.environ, OMP_NUM_THREADS="2")
    t0 = time.time()
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider"] + PIN_TESTS,
                       cwd=tree, env=env, capture_output=True, text=True, timeout=3600)
    el = time.time() - t0
    if r.returncode == 0:
        return name, "SURVIVED", el
    failed = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
    return name, "KILLED " + (failed[0].split(" - ")[0][7:] if failed else "(error)"), el


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workdir", default=None)
    ap.add_argument("--jobs", type=int, default=4)
    ap.add_argument("names", nargs="*")
    args = ap.parse_args()
    with open(os.path.join(ROOT, "oracle", "hji_oracle.c")) as f:
        src = f.read()
    todo = [m for m in MUTATIONS if not args.names or m[0] in args.names]
    workdir = args.workdir or tempfile.mkdtemp(prefix="oracle_mutants_")
    os.makedirs(workdir, exist_ok=True)
    jobs = max(1, min(args.jobs, len(todo)))
    trees = [_tree(workdir, w) for w in range(jobs)]

    def worker(w):
        out = []
        for i in range(w, len(todo), jobs):
            res = _run_one(trees[w], src, todo[i])
            print("%-26s %s (%.0f s)" % res, flush=True)
            out.append(res)
        return out

    with ThreadPoolExecutor(jobs) as ex:
        results = [r for part in ex.map(worker, range(jobs)) for r in part]
    bad = [r[0] for r in results if not r[1].startswith("KILLED")]
    print("%d mutations, %d killed%s" % (len(results), len(results) - len(bad),
                                         (", not killed: " + " ".join(bad)) if bad else ""))
    return 1 if bad else 0


if __name__ == "__main__":
    sys.exit(main())
