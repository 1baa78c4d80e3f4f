"""The user guide's code examples stay valid: the Python example parses, the
C example compiles against include/bgk.h and links to libbgk.so."""
import ast
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _guide():
    """The user guide: the top-level Markdown file that carries the C example."""
    for name in sorted(os.listdir(ROOT)):
        if name.endswith(".md"):
            text = open(os.path.join(ROOT, name)).read()
            if '```c\n#include "bgk.h"' in text:
                return text
    raise AssertionError("no top-level Markdown file carries the C example")


def _blocks(lang):
    return re.findall(r"```%s\n(.*?)```" % lang, _guide(), re.S)


def test_python_example_parses():
    blocks = _blocks("python")
    assert blocks
    for b in blocks:
        ast.parse(b)


def test_c_example_compiles_and_links(tmp_path, libbgk):
    blocks = _blocks("c")
    assert blocks
    body = blocks[0].replace('#include "bgk.h"\n', "")
    src = tmp_path / "example.c"
    src.write_text('#include <stddef.h>\n#include "bgk.h"\nint main(void) {\n'
                   "    const double *q = NULL; double dt = 1e-3;\n" + body + "    return 0;\n}\n")
    libdir = os.path.join(ROOT, "paper_2312_06567_gb300")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir,
                    "-lbgk", "-o", str(tmp_path / "example")], check=True)
