"""Sensitivity of the oracle pins: each plausible mistake, planted in a copy
of the oracle source on the CPU, must make at least one pin fail."""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_partition as tp
from tests import test_oracle_solve as ts

SRC = os.path.join(os.path.dirname(oracle.__file__), "prgb_oracle.c")

MUTANTS = {
    "transposed_power_series": (
        "for (int64_t e = g.iptr[vi]; e < g.iptr[vi + 1]; e++) {\n"
        "                            int32_t j = g.iidx[e];",
        "for (int64_t e = g.optr[vi]; e < g.optr[vi + 1]; e++) {\n"
        "                            int32_t j = g.oidx[e];"),
    "level_update_drops_c": ("W[i] += c * R[j]", "W[i] += R[j]"),
    "one_based_levels": ("level[v] = lvl[h] - 1;", "level[v] = lvl[h];"),
    "scc_does_not_block_merge": ("{ m = 0; break; }", "{ }"),
    "merge_flags_reset_per_edge": (
        "int32_t x = g.oidx[e];\n                            if (vtype[x] == TYPE_SCC",
        "int32_t x = g.oidx[e]; m = 0; nl = 0;\n                            if (vtype[x] == TYPE_SCC"),
    "outdeg_counts_loops": ("g->outdeg[i] = (int32_t)(k - g->optr[i]);",
                            "g->outdeg[i] = (int32_t)(rowptr[i + 1] - rowptr[i]);"),
    "budget_not_split": ("tol * (double)sz / (double)n", "tol"),
    "residual_sign": ("fabs(u[i] + c * s - R[i])", "fabs(u[i] - c * s - R[i])"),
    "tie_break_size_ascending": ("return a->size > b->size ? -1 : 1;",
                                 "return a->size < b->size ? -1 : 1;"),
    "cac_skips_weight": ("R[x] = R[x] + R[w] * (c / (double)g.outdeg[w]);",
                         "R[x] = R[x] + R[w] * c;"),
}

PINS = [
    tp.test_fig1_partition, tp.test_fig1_scc_only_levels,
    tp.test_all_4_vertex_digraphs_match_theorem, tp.test_random_dag_like_digraphs_match_theorem,
    lambda: tp.test_invariants_small_planted(1),
    ts.test_chain_closed_form, lambda: ts.test_cycle_closed_form(7),
    ts.test_out_star, lambda: ts.test_componentwise_converges_to_dense(3),
    lambda: ts.test_dense_oracle_matches_numpy(4), ts.test_mass_conservation_and_budget,
    ts.test_residual_function_closed_form, ts.test_cac_and_singletons_exact_at_loose_tolerance,
]


def _failures(lib_path):
    failed = 0
    with oracle.use_library(lib_path):
        for pin in PINS:
            try:
                pin()
            except (AssertionError, oracle.OracleError):
                failed += 1
    return failed


def test_clean_copy_passes(tmp_path):
    lib = tmp_path / "clean.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", str(lib), SRC, "-lm"])
    assert _failures(str(lib)) == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / f"{name}.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", str(lib), str(mutated), "-lm"])
    assert _failures(str(lib)) >= 1, f"no pin caught the planted mistake {name}"
