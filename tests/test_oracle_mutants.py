"""Plant plausible mistakes in a copy of the oracle (CPU only) and check that
the pins in test_oracle_pins.py catch every one of them."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "density_tie_nonstrict": ("return (i128)e1 * (i128)v2 > (i128)e2 * (i128)v1;",
                              "return (i128)e1 * (i128)v2 >= (i128)e2 * (i128)v1;"),
    "degstar_uses_deg_G": ("int64_t ds = deg[v];                 /* deg*_H(v_j) */",
                           "int64_t ds = off[v + 1] - off[v];"),
    "peel_no_decrement": ("if (inH[adj[e]]) deg[adj[e]] -= 1;", ";"),
    "sort_descending": ("if (lx != ly) return lx < ly ? -1 : 1;", "if (lx != ly) return lx > ly ? -1 : 1;"),
    "sort_ties_by_reverse_id": ("return x < y ? -1 : (x > y ? 1 : 0);", "return x > y ? -1 : (x < y ? 1 : 0);"),
    "round_rule_strict": ("if ((i128)k * q <= (i128)mn * (i128)(p + q)) {",
                          "if ((i128)k * q < (i128)mn * (i128)(p + q) || k == mn) {"),
    "round_rule_eps_dropped": ("if ((i128)k * q <= (i128)mn * (i128)(p + q)) {",
                               "if ((i128)k * q <= (i128)mn * (i128)q) {"),
    "round_key_without_degree": ("int64_t k = loads[v] + deg[v];\n            if ((i128)k",
                                 "int64_t k = loads[v];\n            if ((i128)k"),
    "round_decrement_immediate_skip": ("if (state[adj[e]] == 0) deg[adj[e]] -= 1;", ";"),
    "best_set_off_by_one": ("for (int64_t j = bpos; j < n; ++j) in[border[j]] = 1;",
                            "for (int64_t j = bpos + 1; j < n; ++j) in[border[j]] = 1;"),
    "load_update_dropped": ("loads[v] += ds;                      /* Alg. 2: load update */", ";"),
    "iteration_best_last_max": ("if (ij < 0 || density_gt(eH, vH, ie, iv))",
                                "if (ij < 0 || !density_gt(ie, iv, eH, vH))"),
    "bz_nonstrict": ("if (deg[u] > deg[v]) {", "if (deg[u] >= deg[v]) {"),
    "maxflow_capacity": ("for (int64_t v = 0; v < n; ++v) flow_add(&f, v, t, ga);",
                         "for (int64_t v = 0; v < n; ++v) flow_add(&f, v, t, ga + 1);"),
    "brute_force_double_count": ("if (bm == 0 || density_gt(twice / 2, vs, be, bv)) { be = twice / 2;",
                                 "if (bm == 0 || density_gt(twice, vs, be, bv)) { be = twice;"),
    "deletion_core_off_by_one": ("if (d < k) { in[v] = 0; changed = 1; }", "if (d <= k) { in[v] = 0; changed = 1; }"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(mut)])
    env = dict(os.environ, DSG_ORACLE_SO=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"


# plausible mistakes in the Pruning-and-Refining run (Alg. 1), caught by
# the pins in test_oracle_pruned.py
PRUNE_MUTANTS = {
    "prune_floor_half": ("ceil_div(kmax * c_den, 2 * c_num) : ceil_div(kmax, 2), Ld = 1;",
                         "ceil_div(kmax * c_den, 2 * c_num) : kmax / 2, Ld = 1;"),
    "prune_no_repruning": ("if (nlevel <= level) continue;", "continue;"),
    "prune_loads_reset": ("nl[i] = cl[nold[i]];", "nl[i] = 0;"),
    "prune_L_not_raised": ("if (density_gt(se, sv, Ln, Ld)) { Ln = se; Ld = sv; }", ";"),
    "prune_nonstrict_improvement": ("if (!density_gt(b[0], b[1], se, sv)) continue;",
                                    "if (density_gt(se, sv, b[0], b[1])) continue;"),
    "prune_frozen_loads_dropped": ("if (!cin[i]) loads[old_of[i]] = cl[i];", ";"),
}


# approximate pruning: caught by test_oracle_apx.py
APX_MUTANTS = {
    "apx_levels_shifted": ("return ceil_div(tau * c_num, c_den);", "return ceil_div(tau * c_num, c_den) + 1;"),
    "apx_lower_level": ("while (tau < apx[v]) tau = apx_next_level(tau, c_num, c_den);",
                        "while (apx_next_level(tau, c_num, c_den) <= apx[v]) tau = apx_next_level(tau, c_num, c_den);"),
    "apx_L_without_c": ("ceil_div(kmax * c_den, 2 * c_num) : ceil_div(kmax, 2), Ld = 1;",
                        "ceil_div(kmax, 2) : ceil_div(kmax, 2), Ld = 1;"),
    "apx_exact_cores_in_run": ("int rc = c_num ? oracle_apx_coreness(n, off, adj, c_num, c_den, core) : oracle_coreness(n, off, adj, core);",
                               "int rc = oracle_coreness(n, off, adj, core);"),
    "apx_zero_core_gets_level": ("if (apx[v] == 0) continue;", ";"),
}


def _run_mutant(old, new, test_file, tmp_path, name):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(mut)])
    env = dict(os.environ, DSG_ORACLE_SO=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", test_file)],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(APX_MUTANTS))
def test_apx_pins_catch_mutant(name, tmp_path):
    _run_mutant(*APX_MUTANTS[name], "test_oracle_apx.py", tmp_path, name)


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(PRUNE_MUTANTS))
def test_pruned_pins_catch_mutant(name, tmp_path):
    old, new = PRUNE_MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(mut)])
    env = dict(os.environ, DSG_ORACLE_SO=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pruned.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
