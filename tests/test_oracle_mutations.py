"""The oracle's pins have teeth: plant plausible mistakes in copies of the
oracle (on the CPU) and check that the pin suite fails for each of them.

Each mutant is a one-line text substitution in a copy of oracle/cp_oracle.c,
compiled into a scratch directory together with a copy of the tests.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    # elder rule reversed in H0: the older root dies
    "h0_elder_reversed": (
        "int64_t young = vertex_less(g, ra, rb) ? rb : ra;",
        "int64_t young = vertex_less(g, ra, rb) ? ra : rb;",
    ),
    # first-order tie-break reversed
    "tiebreak_reversed": ("    return a < b;\n}", "    return a > b;\n}"),
    # dual union-find in ascending instead of reversed order (Sec. 3.1)
    "dual_not_reversed": (
        "for (int64_t i = nfacets - 1; i >= 0; --i)",
        "for (int64_t i = 0; i < nfacets; ++i)",
    ),
    # dual pairing with the older representative (Appendix A.4)
    "dual_elder_reversed": (
        "} else if (rkey_less(&rep[ra], &rep[rb])) {",
        "} else if (!rkey_less(&rep[ra], &rep[rb])) {",
    ),
    # the outside vertex treated as the youngest
    "outside_youngest": (
        "if (ra == OUT) {\n            young = rb;",
        "if (ra == OUT) {\n            young = ra;",
    ),
    # wrong death value for H0
    "h0_death_value": (
        "emit(out, cap, n, keep_zero, g->f[young], edges[i].fm,",
        "emit(out, cap, n, keep_zero, g->f[young], g->f[young],",
    ),
    # -0.0 not canonicalised
    "negative_zero": ("f[i] = x == 0.0f ? 0.0f : x;", "f[i] = x;"),
    # birth and death pixels of top pairs swapped
    "top_pixels_swapped": (
        "facets[i].m,\n             rep[young].m, d - 1);",
        "rep[young].m,\n             facets[i].m, d - 1);",
    ),
    # V-filtration with min instead of max over a cell's vertices (Sec. 2.2)
    "cell_value_min": (
        "if (best < 0 || vertex_less(g, best, v)) best = v;",
        "if (best < 0 || vertex_less(g, v, best)) best = v;",
    ),
    # second-order tie-break reversed
    "second_order_reversed": (
        "if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;",
        "if (a->idx != b->idx) return a->idx > b->idx ? -1 : 1;",
    ),
    # zero-persistence filter dropped
    "zero_persistence_kept": (
        "if (!keep_zero && b == d) return 0;",
        "if (0 && b == d) return 0;",
    ),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "cp_oracle.c")).read()
    assert old in src, f"mutant {name} no longer applies to the oracle source"
    d = tmp_path / "repo"
    (d / "oracle").mkdir(parents=True)
    (d / "oracle" / "cp_oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), d / "oracle" / "__init__.py")
    shutil.copytree(os.path.join(ROOT, "tests"), d / "tests", ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copy(os.path.join(ROOT, "workloads.py"), d / "workloads.py")
    r = subprocess.run(
        [sys.executable, "-m", "pytest", str(d / "tests" / "test_oracle_pins.py"), "-x", "-q", "-p", "no:cacheprovider"],
        capture_output=True,
        text=True,
        cwd=str(d),
        timeout=600,
    )
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"


# mistakes in the H1 reduction of volumes, caught by test_oracle_h1_pins.py
H1_MUTANTS = {
    # the pair takes the column's first row instead of its lowest (the youngest)
    "h1_birth_not_lowest": (
        "const rkey *e = &edges[c[nc - 1]];",
        "const rkey *e = &edges[c[0]];",
    ),
    # no column additions: every square keeps its boundary
    "h1_not_reduced": (
        "while (nc > 0 && owner[c[nc - 1]] >= 0) {",
        "while (0 && nc > 0 && owner[c[nc - 1]] >= 0) {",
    ),
    # squares processed from the youngest down
    "h1_columns_reversed": (
        "for (int64_t j = 0; j < nsq; ++j) {",
        "for (int64_t j = nsq - 1; j >= 0; --j) {",
    ),
    # a square's boundary with only the edges on its +1 sides
    "h1_half_boundary": (
        "c[nc++] = erank[(q[0] * g->GH + q[1]) * g->GW + q[2]];",
        "if (s > 0) c[nc++] = erank[(q[0] * g->GH + q[1]) * g->GW + q[2]];",
    ),
    # birth and death values exchanged
    "h1_values_swapped": (
        "emit(out, cap, n, keep_zero, e->fm, sq[j].fm, e->idx, sq[j].idx, e->m, sq[j].m, 1);",
        "emit(out, cap, n, keep_zero, sq[j].fm, e->fm, e->idx, sq[j].idx, e->m, sq[j].m, 1);",
    ),
    # the death pixel taken from the birth edge
    "h1_death_pixel": (
        "emit(out, cap, n, keep_zero, e->fm, sq[j].fm, e->idx, sq[j].idx, e->m, sq[j].m, 1);",
        "emit(out, cap, n, keep_zero, e->fm, sq[j].fm, e->idx, sq[j].idx, e->m, e->m, 1);",
    ),
}


@pytest.mark.parametrize("name", sorted(H1_MUTANTS))
def test_h1_pins_catch_mutant(name, tmp_path):
    old, new = H1_MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "cp_oracle.c")).read()
    assert src.count(old) == 1, f"mutant {name} no longer applies to the oracle source"
    d = tmp_path / "repo"
    (d / "oracle").mkdir(parents=True)
    (d / "oracle" / "cp_oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), d / "oracle" / "__init__.py")
    shutil.copytree(os.path.join(ROOT, "tests"), d / "tests", ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copy(os.path.join(ROOT, "workloads.py"), d / "workloads.py")
    r = subprocess.run(
        [sys.executable, "-m", "pytest", str(d / "tests" / "test_oracle_h1_pins.py"), "-x", "-q", "-p",
         "no:cacheprovider"],
        capture_output=True,
        text=True,
        cwd=str(d),
        timeout=600,
    )
    assert r.returncode != 0, f"mutant {name} survived the H1 pins:\n{r.stdout[-2000:]}"
