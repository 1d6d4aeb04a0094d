"""The pins must be able to fail: plausible mistakes planted in copies of the oracle
source (a swapped link direction, a dropped arc, a wrong index or operand, a missing
reverse arc, a missing final find) must each be caught by the pin set. The mutants
are compiled into a temporary directory and exercised in a child process."""
import os
import subprocess
import sys
import textwrap

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "union_links_smaller_below_larger": (
        "if (ra < rb) parent[rb] = ra;\n  else parent[ra] = rb;",
        "if (ra < rb) parent[ra] = rb;\n  else parent[rb] = ra;"),
    "union_finds_same_operand_twice": (
        "int32_t rb = uf_find(parent, b);", "int32_t rb = uf_find(parent, a);"),
    "csr_drops_last_arc_of_each_row": (
        "a < row_ptr[u + 1]; ++a)\n      uf_union", "a + 1 < row_ptr[u + 1]; ++a)\n      uf_union"),
    "no_final_find": (
        "label[v] = uf_find(label, (int32_t)v);", "label[v] = label[v];"),
    "component_count_inverted": (
        "if (label[v] == v) ++comps;", "if (label[v] != v) ++comps;"),
    "bfs_labels_with_parent_not_source": (
        "label[y] = (int32_t)s;", "label[y] = x;"),
    "bfs_scan_skips_vertex_zero": (
        "for (int64_t s = 0; s < V; ++s) {", "for (int64_t s = 1; s < V; ++s) {"),
    "adjacency_misses_reverse_arc": (
        "g->nbr[fill[head[i]]++] = (int32_t)u;", "g->nbr[fill[head[i]]++] = head[i];"),
}

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {tests!r}); sys.path.insert(0, {root!r})
    import oracle
    from test_oracle_pins import pins
    lib = oracle.load_library({lib!r})
    try:
        pins(lib)
    except (AssertionError, ValueError) as e:
        print("PINS FAILED:", type(e).__name__)
        sys.exit(0)
    print("PINS PASSED")
""")


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutant_src = tmp_path / "oracle_mutant.c"
    mutant_src.write_text(text.replace(old, new))
    lib = oracle.build(force=True, src=str(mutant_src), out=str(tmp_path / "liboracle_mutant.so"))
    code = CHILD.format(tests=os.path.join(ROOT, "tests"), root=ROOT, lib=lib)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert "PINS FAILED" in r.stdout, (name, r.stdout, r.stderr[-2000:])


def test_unmutated_copy_passes(tmp_path):
    lib = oracle.build(force=True, src=SRC, out=str(tmp_path / "liboracle_copy.so"))
    code = CHILD.format(tests=os.path.join(ROOT, "tests"), root=ROOT, lib=lib)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert "PINS PASSED" in r.stdout, (r.stdout, r.stderr[-2000:])
