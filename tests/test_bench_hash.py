"""The source hash that ties the recorded DRAM traffic to the kernel code
ignores comments (host logic of bench.py, no GPU)."""

import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_comments_and_blank_lines_removed():
    b = _bench()
    src = 'int a = 1; // note\n/* block\n comment */ const char *s = "x // y /* z */";\n\nchar c = \'/\';  \n'
    assert b.strip_c_comments(src) == 'int a = 1;\n const char *s = "x // y /* z */";\nchar c = \'/\';'


def test_code_changes_change_the_text():
    b = _bench()
    assert b.strip_c_comments("int a = 1; // x") != b.strip_c_comments("int a = 2; // x")
    assert b.strip_c_comments("int a = 1; // x") == b.strip_c_comments("int a = 1; /* y */")
