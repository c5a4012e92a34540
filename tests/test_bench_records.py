"""The benchmark's kernel-source hash, which ties a committed ncu traffic
record to the code it was taken on (a record of other code is reported as
null): it ignores comments but not code."""
import bench


def test_strip_comments_keeps_code_and_literals():
    src = ('int a = 1; // one\n'
           '/* block\n comment */ int b = 2;\n'
           'const char *s = "not // a comment /* here */";\n'
           "char c = '/';  /* trailing */\n"
           '\n'
           'int d = a / b;  // division stays\n')
    out = bench.strip_comments(src)
    assert out == ('int a = 1;\n'
                   ' int b = 2;\n'
                   'const char *s = "not // a comment /* here */";\n'
                   "char c = '/';\n"
                   'int d = a / b;')


def test_comment_edits_keep_the_hash_code_edits_change_it():
    a = "x = y + 1; // add one\n"
    assert bench.strip_comments(a) == bench.strip_comments("x = y + 1; // plus one\n\n")
    assert bench.strip_comments(a) != bench.strip_comments("x = y + 2; // add one\n")
