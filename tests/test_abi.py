"""CPU checks of the C ABI: the library builds, loads and exports every declared symbol, and
host-side argument checking works without a GPU (no compute call is made)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sx.h")


def _builder():
    import importlib.util
    path = os.path.join(ROOT, "paper_2206_06302_b300", "build.py")
    spec = importlib.util.spec_from_file_location("_sx_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sx_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_and_loads():
    path = _builder().build()
    assert os.path.exists(path)
    import paper_2206_06302_b300 as p
    assert p.sx_version() == 10000


def test_every_declared_symbol_is_exported():
    path = _builder().build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, f"declared but not exported: {missing}"
    assert len(declared_functions()) >= 60


def test_binding_covers_the_header():
    import paper_2206_06302_b300 as p
    assert set(declared_functions()) == set(p.sx.EXPORTED)
    for f in declared_functions():
        assert hasattr(p.sx, f), f


def test_status_strings():
    import paper_2206_06302_b300 as p
    assert p.sx_status_string(p.SX_OK) == "SX_OK"
    assert p.sx_status_string(p.SX_ERR_OVERLAP) == "SX_ERR_OVERLAP"
    assert p.sx_status_string(99) == "SX_ERR_UNKNOWN"


def test_null_handles_are_rejected_without_a_gpu():
    import paper_2206_06302_b300 as p
    with pytest.raises(p.SxError) as ei:
        p.sx_free(None)
    assert ei.value.status == p.SX_ERR_INVALID
    with pytest.raises(p.SxError) as ei:
        p.sx_copy(None, None, None)
    assert ei.value.status == p.SX_ERR_INVALID
    with pytest.raises(p.SxError):
        p.sx_tune_load("/nonexistent/table.json")
    with pytest.raises(p.SxError) as ei:
        p.sx_seed_uniform_at(None, 1, -1.0, 1.0, 5)
    assert ei.value.status == p.SX_ERR_INVALID
    with pytest.raises(p.SxError) as ei:
        p.sx_tune_pass(None, p.SX_F64, 1 << 16)
    assert ei.value.status == p.SX_ERR_INVALID
    with pytest.raises(p.SxError) as ei:
        p.sx_batch_run_noalloc(None, [p.sx_batch_item(op=9, dtype=p.SX_F64, n=1)])
    assert ei.value.status == p.SX_ERR_INVALID  # refused on the host, before any CUDA call


def test_tune_table_roundtrip(tmp_path):
    import paper_2206_06302_b300 as p
    path = tmp_path / "t.json"
    path.write_text('{"ops": [{"device": "X", "op": 3, "dtype": 2, "bucket": 27, "variant": 1,'
                    ' "threads": 512, "blocks_per_sm": 0, "vec_bytes": 32, "unroll": 2,'
                    ' "cache_hint": 1, "tile_bytes": 0, "stages": 0}],'
                    ' "batch": [{"device": "X", "bucket": 20, "chunk_bytes": 262144,'
                    ' "threads": 256, "blocks_per_sm": 4, "vec_bytes": 32}]}')
    p.sx_tune_clear()
    p.sx_tune_load(str(path))
    out = tmp_path / "o.json"
    p.sx_tune_save(str(out))
    s = out.read_text()
    assert '"threads": 512' in s and '"chunk_bytes": 262144' in s and '"device": "X"' in s
    p.sx_tune_clear()


def test_no_device_means_no_target():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2206_06302_b300 as p
    with pytest.raises(p.SxError):
        p.sx_target_create(0)


def build_c_client(tmp_path):
    """Compile and link tests/c_abi_program.c, a plain C11 client, against libsx."""
    lib = _builder().build()
    exe = str(tmp_path / "c_abi_program")
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_program.c"), "-o", exe, "-L", os.path.dirname(lib), "-lsx",
           "-Wl,-rpath," + os.path.dirname(lib)]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


def test_header_is_plain_c_and_links(tmp_path):
    """sx.h compiles as strict C11 and a C client links against libsx; without a device it
    reports that and exits 2 (no compute call is made)."""
    import torch
    exe = build_c_client(tmp_path)
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the GPU test runs the client")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 2 and "no device" in r.stderr, (r.returncode, r.stderr)


def build_cpp_client(tmp_path):
    """Compile and link tests/cpp_api_program.cpp (the header-only C++ layer sx.hpp) against libsx."""
    lib = _builder().build()
    exe = str(tmp_path / "cpp_api_program")
    cmd = ["g++", "-std=c++17", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "cpp_api_program.cpp"), "-o", exe, "-L", os.path.dirname(lib), "-lsx",
           "-Wl,-rpath," + os.path.dirname(lib)]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


def test_cpp_layer_compiles_and_links(tmp_path):
    """sx.hpp compiles as strict C++17 and a client links; without a device it exits 2."""
    import torch
    exe = build_cpp_client(tmp_path)
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the GPU test runs the client")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 2 and "no device" in r.stderr, (r.returncode, r.stderr)


STRUCTS = ["sx_launch_cfg", "sx_target_info", "sx_batch_item", "sx_batch_cfg", "sx_server_cfg",
           "sx_request", "sx_request_status", "sx_server_stats"]


def test_binding_structs_match_the_header(tmp_path):
    """Every public struct of the binding has the header's size and field offsets (a C program
    compiled against sx.h prints them), so a field added on one side only is caught."""
    import ctypes
    from paper_2206_06302_b300 import sx as binding
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sx.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(binding, name)
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name in STRUCTS:
        cls = getattr(binding, name)
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_shipped_tune_table_is_complete_and_valid():
    """The tuner table shipped with the package holds one entry per STREAM kernel, type and log2
    size from 2^16 to 2^29, each a launch shape the library accepts (checked on the host)."""
    import json
    path = os.path.join(ROOT, "paper_2206_06302_b300", "tune_b300.json")
    entries = json.load(open(path))["ops"]
    keys = {(e["op"], e["dtype"], e["bucket"]) for e in entries}
    assert len(keys) == len(entries) == 4 * 2 * 14
    assert keys == {(op, dt, b) for op in range(4) for dt in (1, 2) for b in range(16, 30)}
    for e in entries:
        assert e["variant"] in (1, 2, 3, 4), e
        assert e["threads"] % 32 == 0 and 32 <= e["threads"] <= 1024, e
        assert e["fp64_mul"] in (0, 1, 2), e
        if e["variant"] == 1:
            assert e["vec_bytes"] in (16, 32) and e["unroll"] in (1, 2, 4), e
            assert e["cache_hint"] in (0, 1) and 0 <= e["blocks_per_sm"] <= 64, e
        else:
            assert e["tile_bytes"] % 1024 == 0 and 1024 <= e["tile_bytes"] <= 65536, e
            assert 2 <= e["stages"] <= 8 and 1 <= e["blocks_per_sm"] <= 4, e
            assert e["threads"] >= (96 if e["variant"] in (3, 4) else 64), e
