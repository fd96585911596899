"""Host-side pieces of the benchmark: the kernel-source hash that decides
whether committed ncu traffic figures still describe the kernels."""
import bench


def test_code_only_ignores_comments_and_layout():
    a = 'int f(int x) { return x + 1; }  // add one\n'
    b = '/* add one */\nint f(int x)\n{\n    return x + 1;\n}\n'
    assert bench._code_only(a) == bench._code_only(b)


def test_code_only_keeps_code_and_literals():
    base = bench._code_only('int f(int x) { return x + 1; }')
    assert bench._code_only('int f(int x) { return x + 2; }') != base
    # comment markers inside string and character literals are code
    s = bench._code_only('const char *p = "a // b /* c */"; char q = \'/\'; // tail')
    assert s == 'const char *p = "a // b /* c */"; char q = \'/\';'
    e = bench._code_only('const char *p = "say \\"hi\\" // not a comment";')
    assert e == 'const char *p = "say \\"hi\\" // not a comment";'


def test_csrc_hash_is_stable():
    assert bench.csrc_hash() == bench.csrc_hash()
    assert len(bench.csrc_hash()) == 16
