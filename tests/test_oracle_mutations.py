"""The oracle's pins catch plausible mistakes (CPU only).

Each case copies ipgc_oracle.c, plants one mistake by a textual edit,
compiles the copy into a temporary library and runs the hand-worked and
closed-form pins against it: at least one pin must fail. This shows the pins
constrain the parts of Section II-C a slip would most likely break.
"""
import itertools
import os
import subprocess

import numpy as np
import pytest

import oracle
from test_oracle_pins import csr_from_edges, load_golden

SRC = os.path.join(os.path.dirname(oracle.__file__), "ipgc_oracle.c")

MUTATIONS = {
    # the lower ID loses a conflict instead of the higher one
    "tie_rule_flipped": ("if (active[u] && u < v && T[u] == T[v])",
                         "if (active[u] && u > v && T[u] == T[v])"),
    # colours written during step 1 (no snapshot: Gauss-Seidel reads)
    "no_snapshot": ("      T[v] = t;\n", "      T[v] = t;\n      color[v] = t;\n"),
    # first fit starts at 2 instead of 1
    "mex_from_2": ("int32_t t = 1;", "int32_t t = 2;"),
    # a dropped term in the conflict test: conflicts with node 0 are missed
    "skip_node_zero": ("if (active[u] && u < v && T[u] == T[v])",
                       "if (active[u] && u < v && u != 0 && T[u] == T[v])"),
    # the colour bound ignores colour deg+1 and colour 1
    "ignore_colour_1": ("if (c >= 1 && c <= deg + 1)", "if (c >= 2 && c <= deg + 1)"),
    # the final conflict-free round is not counted
    "round_count": ("  *rounds_out = round;", "  *rounds_out = round - 1;"),
}


def pins_pass(lib):
    for name in ("handworked_g7.txt", "handworked_g8.txt"):
        n, edges, colors, rounds, k, wl = load_golden(name)
        res = oracle.color(*csr_from_edges(n, edges), lib=lib)
        if not (np.array_equal(res.colors, colors) and res.rounds == rounds and res.num_colors == k):
            return False
    for n in (3, 6):
        res = oracle.color(*csr_from_edges(n, list(itertools.combinations(range(n), 2))), lib=lib)
        if not (np.array_equal(res.colors, np.arange(1, n + 1)) and res.rounds == n):
            return False
    for n in (4, 7):
        res = oracle.color(*csr_from_edges(n, [(i, i + 1) for i in range(n - 1)]), lib=lib)
        if not (np.array_equal(res.colors, np.array([1 + i % 2 for i in range(n)])) and res.rounds == n // 2 + 1):
            return False
    res = oracle.color(*csr_from_edges(5, [(0, i) for i in range(1, 5)]), lib=lib)
    if not (res.colors.tolist() == [1, 2, 2, 2, 2] and res.rounds == 2):
        return False
    return True


def test_unmutated_passes():
    assert pins_pass(oracle._load())


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(mutant)], check=True)
    assert not pins_pass(oracle.load_library(str(so))), name
