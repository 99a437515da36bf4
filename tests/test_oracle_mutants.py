"""The oracle's pins have teeth: each plausible mistake, planted in a copy of
the oracle's C source on the CPU, fails at least one pin."""
import os

import pytest

import oracle
import oracle_pins as pins

MUTANTS = {
    "cell_index_transposed": ("9 * a + 3 * b + d", "3 * a + 9 * b + d"),
    "dropped_plus_one": ("lf[r0 + r1 + 1] - lf[r0]", "lf[r0 + r1] - lf[r0]"),
    "wrong_sign": (") - lf[r1];", ") + lf[r1];"),
    "dropped_term": ("(lf[r0 + r1 + 1] - lf[r0]) - lf[r1]", "lf[r0 + r1 + 1] - lf[r0]"),
    "classes_swapped": ("ft[c * NCELL + 9", "ft[(1 - c) * NCELL + 9"),
    "log_shifted": ("log((double)n)", "log((double)(n + 1))"),
    "highest_wins": ("return a->k2 < b->k2;", "return a->k2 > b->k2;"),
    "tiebreak_reversed": ("return a->i < b->i;", "return a->i > b->i;"),
    "last_sample_dropped": ("s < n_samples; ++s", "s + 1 < n_samples; ++s"),
    "k_loop_skips": ("int32_t k = j + 1;", "int32_t k = j + 2;"),
    "pair_cell_transposed": ("ft[c * NPCELL + 3 * a + b]", "ft[c * NPCELL + a + 3 * b]"),
    "pair_classes_swapped": ("ft[c * NPCELL + 3 * a + b] += 1;",
                             "ft[(1 - c) * NPCELL + 3 * a + b] += 1;"),
    "pair_last_cell_skipped": ("cell < NPCELL; ++cell", "cell < NPCELL - 1; ++cell"),
    "order_digits_reversed": ("cell = 3 * cell + g;", "cell = cell + g * cells_of(t);"),
    "order_classes_swapped": ("ft[c * ncell + cell] += 1;", "ft[(1 - c) * ncell + cell] += 1;"),
    "order_dropped_plus_one": ("double term = (lf[r0 + r1 + 1] - lf[r0]) - lf[r1];\n        k2 = k2 + term;\n    }\n    return k2;\n}\n\n/* Tables of n SNP sets",
                               "double term = (lf[r0 + r1] - lf[r0]) - lf[r1];\n        k2 = k2 + term;\n    }\n    return k2;\n}\n\n/* Tables of n SNP sets"),
    "order_last_snp_skips": ("if (x[depth] > n_snps - (order - depth)) {",
                             "if (x[depth] > n_snps - (order - depth) - 1) {"),
    "order_tiebreak_reversed": ("if (a->x[t] != b->x[t]) return a->x[t] < b->x[t];",
                                "if (a->x[t] != b->x[t]) return a->x[t] > b->x[t];"),
    "pair_j_loop_skips": ("for (int32_t j = i + 1; j < n_snps; ++j) {\n                int32_t ft[2 * NPCELL];",
                          "for (int32_t j = i + 2; j < n_snps; ++j) {\n                int32_t ft[2 * NPCELL];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    before, after = MUTANTS[name]
    with open(oracle._SRC) as f:
        src = f.read()
    assert before in src, f"mutation site for {name} not found"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(before, after, 1))
    lib = oracle.build(force=True, src=str(path), out=str(tmp_path / f"lib{name}.so"))
    o = oracle.Oracle(lib)
    caught = []
    for check in pins.ALL_CHECKS:
        try:
            check(o)
        except (AssertionError, ValueError):
            caught.append(check.__name__)
    assert caught, f"no pin catches the {name} mutant"
