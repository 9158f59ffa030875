"""bench.py reports the DRAM traffic of the single-solve kernels from a
committed ncu record only while the kernels' code is the code it was taken
on. The hash that decides this ignores comments and layout, and must change
with any change to the code itself (CPU only)."""

import bench

SRC = """// a leading comment
__global__ void k(int *a, int n) {   /* trailing
   block comment */
    int i = threadIdx.x;  // index
    if (i < n) a[i] = 2 * i;
}
"""


def test_comments_and_layout_do_not_count():
    edited = SRC.replace("// index", "// the lane's index").replace("a leading", "another")
    relaid = SRC.replace("    int i", "\tint  i").replace("\n}", "\n\n}")
    assert bench.code_tokens(edited) == bench.code_tokens(SRC)
    assert bench.code_tokens(relaid) == bench.code_tokens(SRC)
    assert "comment" not in bench.code_tokens(SRC) and "index" not in bench.code_tokens(SRC)


def test_code_changes_count():
    for old, new in (("2 * i", "3 * i"), ("i < n", "i <= n"), ("int *a", "long *a")):
        assert bench.code_tokens(SRC.replace(old, new)) != bench.code_tokens(SRC)


def test_hashed_sources_hold_no_comment_marker_in_a_string():
    """The stripper does not parse string literals; the hashed files must not
    need it to."""
    import os
    import re
    csrc = os.path.join(bench.ROOT, "paper_1110_6231_gb300", "csrc")
    for name in bench.SINGLE_SOLVE_SOURCES:
        text = open(os.path.join(csrc, name)).read()
        assert not re.search(r'"[^"\n]*(//|/\*)[^"\n]*"', text), name


def test_every_single_solve_line_finds_its_traffic_record():
    """Each full bench line reports roofline.traffic from a record taken on
    its own workload, alpha and solver options and on the kernel code built
    now: a kernel change without a new capture shows up here, not as a null
    in the next bench line."""
    roles = {"uniform-n256-c1000": ("k_small",)}
    for workload, spec in bench.LINES.items():
        for kernel in roles.get(workload, ("k_refine_sweep", "k_refine", "k_tail")):
            got = bench.recorded_traffic(workload, spec["alpha"], kernel, spec.get("options"))
            assert got is not None and got > 0, (workload, kernel)


def test_bench_line_options_are_solver_options():
    """bench.py sets each line's options on la_options by name; a ctypes
    structure would silently take a misspelt name as a new attribute, so
    every name must be one of the structure's fields."""
    import paper_1110_6231_gb300 as la
    fields = {name for name, _ in la.la_options._fields_}
    for workload, spec in bench.LINES.items():
        for name in spec.get("options", {}):
            assert name in fields, (workload, name)
