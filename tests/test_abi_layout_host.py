"""The ctypes binding's structs against the C header's layout: every field of
henry_config, henry_tuning and henry_stats at the same offset and the same
size, and the same struct sizes, as a C compiler lays them out from
include/henry.h (a small program built with the host compiler prints them).
A field added to one side only, or in another order, fails here instead of
shifting every later field in the library's view."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _layout_program(structs):
    lines = ["#include <stddef.h>", "#include <stdio.h>", "#include \"henry.h\"", "int main(void) {"]
    for cname, fields in structs:
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in fields:
            lines.append('  printf("%s %s %%zu %%zu\\n", offsetof(%s, %s), sizeof(((%s*)0)->%s));'
                         % (cname, f, cname, f, cname, f))
    lines += ["  return 0;", "}"]
    return "\n".join(lines) + "\n"


def test_binding_structs_match_the_header_layout(tmp_path):
    import ctypes
    from paper_2302_07804_gb300 import henry
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    structs = [("henry_config", henry.HenryConfig), ("henry_tuning", henry.HenryTuning),
               ("henry_stats", henry.HenryStats)]
    src = tmp_path / "layout.c"
    src.write_text(_layout_program([(c, [n for n, _ in s._fields_]) for c, s in structs]))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        parts = line.split()
        if len(parts) == 3 and parts[1] == "sizeof":
            got[(parts[0], "sizeof")] = int(parts[2])
        elif len(parts) == 4:
            got[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    for cname, s in structs:
        assert got[(cname, "sizeof")] == ctypes.sizeof(s), cname
        for name, ctype in s._fields_:
            field = getattr(s, name)
            assert got[(cname, name)] == (field.offset, ctypes.sizeof(ctype)), (cname, name)
