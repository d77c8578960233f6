"""The kernel-code hash that ties the committed DRAM traffic per entry to
the kernel source: comments and layout do not change it, code does, and
string literals are kept whole (a "//" inside one is code, not a comment)."""
import bench

SRC = '''// header comment
#include "x.h"  /* trailing */
__device__ int f(int a) {   // what f does
  const char *s = "a // b /* c */";
  return a + 1;  /* one
                    two */
}
'''


def test_comments_and_layout_do_not_count():
    edited = SRC.replace("// what f does", "// f adds one").replace("/* trailing */", "")
    edited = edited.replace("  return a + 1;", "      return a + 1;\n\n")
    assert bench.code_only(edited) == bench.code_only(SRC)


def test_code_and_literals_count():
    assert bench.code_only(SRC.replace("a + 1", "a + 2")) != bench.code_only(SRC)
    assert '"a // b /* c */"' in bench.code_only(SRC)
    assert "header" not in bench.code_only(SRC) and "two" not in bench.code_only(SRC)


def test_hash_reads_both_kernel_sources():
    files = {"step_impl.cuh": SRC, "lbm_internal.h": "int k;"}
    h = bench.kernel_source_hash(files.__getitem__)
    assert len(h) == 16
    files["lbm_internal.h"] = "int k; // a note"
    assert bench.kernel_source_hash(files.__getitem__) == h
    files["lbm_internal.h"] = "int k2;"
    assert bench.kernel_source_hash(files.__getitem__) != h
