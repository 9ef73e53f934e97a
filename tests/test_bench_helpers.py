"""Host-side helpers of bench.py: the kernel-source hash that ties the
committed DRAM-traffic figure to the code it was captured on."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_code_only_drops_comments_and_spacing():
    b = _bench()
    a = "int x = 1; // one\n/* block\n comment */ float y;\n"
    c = "int x = 1;\n\n   float y; // another note\n"
    assert b._code_only(a) == b._code_only(c) == "int x = 1; float y;"
    # code changes still change the text that is hashed
    assert b._code_only("int x = 2;") != b._code_only("int x = 1;")


def test_kernel_source_hash_is_stable():
    b = _bench()
    h = b.kernel_source_hash()
    assert len(h) == 16 and h == b.kernel_source_hash()
