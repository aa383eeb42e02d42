"""The C-ABI library builds, loads and exports what include/axlbm.h declares.

CPU only: no call here launches GPU work.  The struct layouts of the ctypes
binding are checked against the header by compiling a tiny C program with gcc.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "axlbm.h")


@pytest.fixture(scope="module")
def built():
    from paper_1003_0282_gb300 import build
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("no CUDA toolkit to build the library")
    return build.build()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"AXLBM_API\s+[\w\s\*]+?\b(axlbm_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for need in ("axlbm_create", "axlbm_step", "axlbm_moments", "axlbm_residual", "axlbm_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (axlbm_\w+)", out))
    assert exported == set(declared_symbols())


def test_binding_struct_layout_matches_header(tmp_path):
    from paper_1003_0282_gb300 import axlbm as B
    prog = tmp_path / "sizes.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "axlbm.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(axlbm_grid), sizeof(axlbm_forcing),"
        " sizeof(axlbm_boundary), offsetof(axlbm_grid, r0), offsetof(axlbm_boundary, r_split),"
        " offsetof(axlbm_boundary, t_wall)); return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(B.axlbm_grid), ctypes.sizeof(B.axlbm_forcing), ctypes.sizeof(B.axlbm_boundary),
            B.axlbm_grid.r0.offset, B.axlbm_boundary.r_split.offset, B.axlbm_boundary.t_wall.offset]
    assert got == want


def test_checkpoint_header_layout_matches_binding(tmp_path):
    """The library's checkpoint header (csrc/internal.h) against the binding's reader and the
    offsets include/axlbm.h documents."""
    from paper_1003_0282_gb300 import axlbm as B
    from paper_1003_0282_gb300 import build
    try:
        cuda_include = os.path.join(os.path.dirname(os.path.dirname(build.nvcc())), "include")
    except RuntimeError:
        pytest.skip("no CUDA toolkit headers")
    fields = [name for name, _, _ in B.CHECKPOINT_HEADER]
    member = {"time": "t"}
    prog = tmp_path / "ckpt.cpp"
    prog.write_text(
        '#include <cstdio>\n#include <cstddef>\n#include "internal.h"\nint main(){\n'
        '  printf("%zu", sizeof(axl::CkptHeader));\n'
        + "".join(f'  printf(" %zu", offsetof(axl::CkptHeader, {member.get(f, f)}));\n' for f in fields)
        + '  printf(" %u %u %u\\n", axl::kCkptVersion, axl::kCkptDomain, axl::kCkptBatch);\n  return 0;\n}\n')
    exe = tmp_path / "ckpt"
    subprocess.run(["g++", "-std=c++17", "-I", os.path.join(ROOT, "paper_1003_0282_gb300", "csrc"), "-I",
                    cuda_include, str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got[0] == B.CHECKPOINT_HEADER_BYTES == 64
    assert got[1:1 + len(fields)] == [off for _, off, _ in B.CHECKPOINT_HEADER]
    assert got[1 + len(fields):] == [1, 1, 2]


def test_host_only_calls(built):
    from paper_1003_0282_gb300 import axlbm as B
    assert B.axlbm_abi_version() == 5
    g = B.axlbm_grid(nr=100, nz=37, precision=B.FP32, with_swirl=1, with_temperature=0, collision=0, r0=0.0)
    n = B.axlbm_state_bytes(g)
    assert n >= 13 * 37 * 128 * 4  # 13 planes, rows padded to 128 floats
    g.nr = 0
    with pytest.raises(B.AxlbmError) as ei:
        B.axlbm_state_bytes(g)
    assert ei.value.status == B.EINVAL
    g.nr, g.precision = 10, 9
    with pytest.raises(B.AxlbmError):
        B.axlbm_state_bytes(g)
    # checkpoint calls without a handle are refused before any device work
    L, n = B.lib(), ctypes.c_size_t(0)
    for save in (L.axlbm_save, L.axlbm_batch_save):
        assert save(None, None, 0, ctypes.byref(n)) == B.EINVAL
    for load in (L.axlbm_load, L.axlbm_batch_load):
        assert load(None, None, 0) == B.EINVAL


def test_create_rejects_invalid_problems_before_any_device_work(built):
    """Validation runs on the host before the first CUDA call."""
    from paper_1003_0282_gb300 import axlbm as B
    from paper_1003_0282_gb300 import inputs as I

    def attempt(**change):
        pb = I.Problem(nr=8, nz=8, tau=0.8, **{k: v for k, v in change.items() if k != "tau_arg"})
        g, tau, f, b = B.structs(pb, "fp32")
        if "tau_arg" in change:
            tau = change["tau_arg"]
        with pytest.raises(B.AxlbmError) as ei:
            B.axlbm_create(g, tau, f, b)
        return ei.value.status

    assert attempt(tau_arg=0.5) == B.EINVAL
    assert attempt(r0=1.0) == B.EINVAL                       # axis needs r0 == 0
    assert attempt(z_lo="wall") == B.EINVAL                  # one periodic face
    assert attempt(z_lo="mixed", z_hi="wall") == B.EINVAL    # mixed bottom
    assert attempt(rho0=-1.0) == B.EINVAL
    assert attempt(temperature=True, tau_t=0.4) == B.EINVAL
