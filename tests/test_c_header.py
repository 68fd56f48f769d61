"""include/dvqls.h is a plain C interface: it compiles as C99 and as C++17
with warnings as errors, and a C program that takes the address of every
function it declares links against libdvqls.so and runs.  The only calls the
program makes are dvqls_create -- without a GPU it returns an error status
instead of crashing; with one it gives a context, which is destroyed again --
and dvqls_last_error on a NULL context, which still returns a string.  No
compute call is made."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")
OUT = os.path.join(ROOT, "paper_2604_14435_gb300", "_build", "c_abi_check")


def declared_functions():
    txt = open(os.path.join(INC, "dvqls.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return re.findall(r"^[A-Za-z_].*?\b(dvqls_\w+)\s*\(", txt, re.M)


def compiler(name):
    path = shutil.which(name)
    if path is None:
        pytest.skip(name + " not found")
    return path


def run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, " ".join(cmd) + "\n" + r.stdout + r.stderr
    return r.stdout


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2604_14435_gb300 import dvqls
    os.makedirs(OUT, exist_ok=True)
    return dvqls.LIB_PATH


@pytest.mark.parametrize("lang", ["c99", "c++17"])
def test_header_compiles_alone(lang):
    os.makedirs(OUT, exist_ok=True)
    ext = "c" if lang == "c99" else "cpp"
    src = os.path.join(OUT, "header_only." + ext)
    with open(src, "w") as f:
        f.write('#include "dvqls.h"\nint dvqls_header_check(void) { return DVQLS_OK; }\n')
    cc = compiler("gcc" if lang == "c99" else "g++")
    run([cc, "-std=" + lang, "-Wall", "-Wextra", "-Werror", "-pedantic", "-I" + INC, "-fsyntax-only", src])


def test_c_program_links_every_function(built):
    names = declared_functions()
    assert len(set(names)) == len(names) and len(names) >= 20
    src = os.path.join(OUT, "link_all.c")
    exe = os.path.join(OUT, "link_all")
    table = ",\n".join("    (fn)%s" % n for n in names)
    with open(src, "w") as f:
        f.write("#include <stdio.h>\n#include \"dvqls.h\"\n"
                "typedef void (*fn)(void);\n"
                "static fn const table[] = {\n%s\n};\n"
                "int main(void) {\n"
                "    size_t i, n = sizeof table / sizeof table[0];\n"
                "    dvqls_ctx* h = NULL;\n"
                "    int rc;\n"
                "    for (i = 0; i < n; ++i)\n"
                "        if (!table[i]) return 2;\n"
                "    rc = dvqls_create(&h, 0, NULL);\n"
                "    printf(\"%%d %%lu %%d\\n\", rc, (unsigned long)n, dvqls_last_error(NULL) != NULL);\n"
                "    if (rc == DVQLS_OK) dvqls_destroy(h);\n"
                "    return 0;\n"
                "}\n" % table)
    libdir = os.path.dirname(built)
    run([compiler("gcc"), "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I" + INC, src, "-o", exe,
         "-L" + libdir, "-ldvqls", "-Wl,-rpath," + libdir, "-Wl,-rpath-link,/usr/local/cuda/lib64"])
    rc, n, has_msg = (int(v) for v in run([exe]).split())
    assert n == len(names) and has_msg == 1
    import torch
    if torch.cuda.is_available():
        assert rc == 0
    else:
        assert rc != 0
