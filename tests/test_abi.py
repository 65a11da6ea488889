"""The C-ABI library builds for sm_103a and exports every entry point that
include/gb300_eri.h declares (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "gb300_eri.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol():
    from paper_2412_13203_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    names = declared()
    assert len(names) >= 10
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    import paper_2412_13203_gb300 as g
    assert sorted(g.EXPORTS) == names


def test_library_loads_and_reports_errors():
    import ctypes
    import paper_2412_13203_gb300 as g
    lib = g.load()
    for n in declared():
        assert hasattr(lib, n)
    # a host-only failure path: a null handle is rejected with a message
    rc = lib.shellpairs_info(None, None, None, None, None)
    assert rc == -1 and b"null" in lib.jk_last_error()
    assert lib.jk_set_option(0, -1.0) == -1


def test_header_is_plain_c_and_links(tmp_path):
    """A C99 program includes the header, links the library and calls host-only
    entry points (no GPU needed): the boundary is usable without C++ or torch."""
    from paper_2412_13203_gb300 import build
    lib = build.build()
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "gb300_eri.h"
int main(void) {
    int lmax = -1, glmax = -1;
    double tau = 0.0;
    if (jk_limits(&lmax, &glmax) != JK_OK) return 1;
    if (jk_get_option(JK_OPT_MIXED_TAU, &tau) != JK_OK) return 2;
    if (shellpairs_info(NULL, NULL, NULL, NULL, NULL) != JK_ERR_INVALID) return 3;
    if (strlen(jk_last_error()) == 0) return 4;
    printf("%d %d %g\n", lmax, glmax, tau);
    return 0;
}
''')
    exe = tmp_path / "use"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"), str(src),
                    lib, "-o", str(exe), f"-Wl,-rpath,{os.path.dirname(lib)}"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out
    assert out.stdout.split() == ["3", "3", "0.005"]


def test_binding_option_names_match_the_header():
    """The Python binding's option table names every jk_option of the header
    with its value (a renumbered or added option cannot drift apart)."""
    import re
    import paper_2412_13203_gb300 as g
    text = open(os.path.join(ROOT, "include", "gb300_eri.h")).read()
    body = text[text.index("typedef enum {", text.index("JK_OPT_MIXED_TAU") - 200):text.index("} jk_option;")]
    enum = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"JK_OPT_(\w+) = (\d+)", body)}
    assert enum and enum == g.JK_OPT
