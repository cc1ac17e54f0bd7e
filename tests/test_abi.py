"""The C-ABI library loads and exports every entry point include/rbfgb.h
declares; argument validation that needs no GPU answers with a status."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2509_26222_gb300 import build as B


def declared():
    names = set()
    for fn in os.listdir(B.INC):
        if fn.endswith(".h"):
            txt = open(os.path.join(B.INC, fn)).read()
            names |= set(re.findall(r"^\s*(?:rbf_status|const char\*)\s+(rbf_\w+)\s*\(", txt, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 16
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rbf_\w+)", out))
    assert names <= exported, names - exported
    for n in names:
        getattr(lib, n)


def test_config_validation_without_gpu():
    from paper_2509_26222_gb300 import native as N
    lib = N.load()
    cfg = N.RbfConfig()
    cfg.kernel = 7
    cfg.lambda_ = 1e-3
    cfg.rho = 0.6
    h = ctypes.c_void_p()
    st = lib.rbf_create(ctypes.byref(cfg), ctypes.byref(h))
    assert st == -1 and b"kernel" in lib.rbf_last_error()
    cfg.kernel = 0
    cfg.lambda_ = 0.0
    st = lib.rbf_create(ctypes.byref(cfg), ctypes.byref(h))
    assert st == -1 and b"lambda" in lib.rbf_last_error()
    assert lib.rbf_destroy(None) == 0


def test_struct_layout_matches_header(tmp_path):
    """ctypes mirror of rbf_config has the offsets a C compiler gives the header."""
    from paper_2509_26222_gb300 import native as N
    fields = [f[0] for f in N.RbfConfig._fields_]
    cname = {"lambda_": "lambda"}
    src = tmp_path / "layout.c"
    body = "".join(f'printf("%zu\\n", offsetof(rbf_config, {cname.get(f, f)}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rbfgb.h"\n'
                   'int main(void){' + body + 'printf("%zu\\n", sizeof(rbf_config)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", B.INC, str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals[:-1] == [getattr(N.RbfConfig, f).offset for f in fields]
    assert vals[-1] == ctypes.sizeof(N.RbfConfig)
