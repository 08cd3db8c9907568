"""bench.py's host logic (no GPU): the ncu traffic record applies while the code of the
sources k_batch is compiled from is unchanged, comments aside."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_text_drops_comments_and_layout():
    src = ('// the row\'s "pivot"\n'
           'int  a = 1;   /* block\n  comment */  int b = 2; // trailing\n'
           '\n\n'
           'const char* s = "x // not a comment /* nor this */";\n'
           "char q = '\\'';  char r = '\"';\n"
           'asm("add %0;\\n" : "=r"(a));\n')
    assert bench.code_text(src) == ('int a = 1;\n'
                                    'int b = 2;\n'
                                    'const char* s = "x // not a comment /* nor this */";\n'
                                    "char q = '\\''; char r = '\"';\n"
                                    'asm("add %0;\\n" : "=r"(a));')


def test_digest_ignores_comments_not_code():
    files = {"a.cu": "int f(int x) { return x + 1; }  // one more\n",
             "b.h": "/* header */\n#define N 4\n"}
    base = bench.sources_sha256(("a.cu", "b.h"), read=files.__getitem__)
    reflowed = {"a.cu": "// a new comment\nint f(int x) {   return x + 1; }\n",
                "b.h": "#define N 4   /* four */\n\n"}
    assert bench.sources_sha256(("a.cu", "b.h"), read=reflowed.__getitem__) == base
    changed = {"a.cu": "int f(int x) { return x + 2; }\n", "b.h": files["b.h"]}
    assert bench.sources_sha256(("a.cu", "b.h"), read=changed.__getitem__) != base
    # the file boundary counts: code moved from one file to the next changes the digest
    moved = {"a.cu": "int f(int x) { return x + 1; }\n#define N 4\n", "b.h": ""}
    assert bench.sources_sha256(("a.cu", "b.h"), read=moved.__getitem__) != base


def test_traffic_record_only_for_the_bench_grid():
    assert bench.recorded_traffic(bench.GRID // 2) is None
