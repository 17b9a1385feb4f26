"""Host-side checks of the benchmark's bookkeeping (no GPU): the recorded DRAM traffic of a
kernel stays attached to its code, not to its comments."""

import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_strip_comments_keeps_code_and_literals():
    b = load_bench()
    src = 'int a = 1;  // note\n/* block\n comment */ const char *s = "x // y /* z */";\nchar q = \'"\'; int c;'
    got = b.strip_comments(src)
    assert got == 'int a = 1; const char *s = "x // y /* z */"; char q = \'"\'; int c;'
    # a comment or layout change leaves the text alone; a code change does not
    assert b.strip_comments(src.replace("// note", "// another note").replace("  ", " ")) == got
    assert b.strip_comments(src.replace("a = 1", "a = 2")) != got

