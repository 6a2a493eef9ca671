"""Host-only checks of the C ABI: the library builds for sm_103a, loads, and exports
every function include/ssilvb.h declares.  No compute call is made (no GPU here)."""
import ctypes
import os
import re

import pytest

import paper_2301_11376_gb300 as ssilvb

HEADER = os.path.join(ssilvb.INCLUDE, "ssilvb.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ssilvb_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    ssilvb.build()
    return ssilvb.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for want in ("ssilvb_create", "ssilvb_gather", "ssilvb_destroy", "ssilvb_gather_host", "ssilvb_synchronize",
                 "ssilvb_status_string", "ssilvb_last_error", "ssilvb_version"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_status_strings(lib):
    for code, name in ssilvb.STATUS_NAMES.items():
        expect = "SSILVB_OK" if code == 0 else "SSILVB_ERR_" + name
        assert lib.ssilvb_status_string(code).decode() == expect
    assert lib.ssilvb_version() >= 10000


def test_struct_layouts_match_header(tmp_path):
    """Every ctypes mirror has the size and field offsets the C compiler gives the header."""
    import subprocess
    mirrors = {"ssilvb_gbuffer": ssilvb.Gbuffer, "ssilvb_camera": ssilvb.CameraC, "ssilvb_params": ssilvb.ParamsC,
               "ssilvb_output": ssilvb.Output, "ssilvb_tuning": ssilvb.Tuning, "ssilvb_frame": ssilvb.Frame}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ssilvb.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", ssilvb.INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            parts = line.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_null_arguments_rejected_without_gpu(lib):
    assert lib.ssilvb_create(None, 0) == 1
    assert lib.ssilvb_gather(None, None, None, None, None, None) == 1
    assert lib.ssilvb_destroy(None) == 0
