"""CPU-side checks of the boundary: the library builds, loads and exports every
symbol declared in include/bie2d.h; the binding's structs match the header.
No compute call is made (there may be no GPU)."""
import ctypes
import re
import subprocess

import pytest

from paper_1507_05925_gb300 import bie, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return bie.load()


def test_exports_every_declared_symbol(lib):
    names = bie.declared_symbols()
    assert set(names) >= {"bie_create", "bie_destroy", "bie_last_error", "elastance_solve",
                          "mobility_solve", "apply_operator", "bie_profile", "bie_server_create",
                          "bie_server_submit", "bie_server_wait", "bie_server_destroy", "bie_workspace_bytes"}
    for n in names:
        assert hasattr(lib, n), n


def _header_struct_fields(name):
    text = open(build.INCLUDE + "/bie2d.h").read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", text, flags=re.S).group(1)
    return re.findall(r"(\w+)\s*;", body.replace("*", " "))


@pytest.mark.parametrize("cname,pyclass", [("bie_geometry", bie.BieGeometry), ("bie_opts", bie.BieOpts),
                                           ("bie_info", bie.BieInfo)])
def test_binding_structs_match_header(cname, pyclass):
    fields = _header_struct_fields(cname)
    assert fields == [f for f, _ in pyclass._fields_]


def test_struct_layout_matches_c_compiler(tmp_path):
    # sizes and field offsets as the C compiler lays them out from the header
    checks = []
    structs = (("bie_geometry", bie.BieGeometry), ("bie_opts", bie.BieOpts), ("bie_info", bie.BieInfo),
               ("bie_profile_counters", bie.BieProfileCounters), ("bie_request", bie.BieRequest))
    for cname, cls in structs:
        checks.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            checks.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"bie2d.h\"\nint main(void){"
                   + "".join(checks) + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", build.INCLUDE, str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    for cname, cls in structs:
        assert int(got[cname]) == ctypes.sizeof(cls)
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.bie_create(ctypes.byref(h), 0, 0)
    assert rc == bie.ERR_CUDA and not h.value


def test_new_entry_points_reject_bad_arguments_without_a_gpu(lib):
    # argument checks come before any CUDA call: no context, no count, no server
    geo = (bie.BieGeometry * 1)()
    ptrs = (ctypes.c_void_p * 1)()
    infos = (bie.BieInfo * 1)()
    status = (ctypes.c_int32 * 1)()
    for fn in (lib.elastance_solve_batch, lib.mobility_solve_batch):
        assert fn(None, 1, geo, ptrs, ptrs, None, infos, status, None) == bie.ERR_INVALID
    S, ms = ctypes.c_int32(), ctypes.c_double()
    assert lib.bie_tune(None, None, 0, 1, ctypes.byref(S), ctypes.byref(ms), None) == bie.ERR_INVALID
    lib.bie_tune_clear()  # host-side table only
    assert lib.bie_server_batching(None, 8, 0, None) == bie.ERR_INVALID
