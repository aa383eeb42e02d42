"""The C ABI's host code under AddressSanitizer and UndefinedBehaviorSanitizer.

The library's sources are compiled with the host parts instrumented
(-fsanitize=address and undefined via nvcc's host compiler).  The device
parts are emitted as PTX only, since nothing here runs on a GPU.  A
subprocess with the ASan runtime preloaded then drives every host path that
needs no device:
- every entry point with NULL handles and zero arguments, which must answer
  AXLBM_EINVAL;
- the device-layout calculation of single domains over random and invalid
  grids;
- the batch planner (shelf packing, tile lists of every candidate shape, ring
  and wall lists, offsets) on the full sweep in both storages and on random
  uneven domain lists;
- problem validation in axlbm_create.

Any memory error or undefined behaviour ends the subprocess with a report.
CPU only.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(ROOT, "include", "axlbm.h")

DRIVER = r"""
import ctypes, re, sys
import numpy as np
sys.path[:0] = [{root!r}, {tests!r}]
from paper_1003_0282_gb300 import axlbm as B, inputs as I
from parity_util import BOUNDARY_MIXES, problem
B.LIB_PATH = {lib!r}
L = B.lib()

# every entry point with NULL handles and zero arguments
names = sorted(set(re.findall(r"AXLBM_API\s+[\w\s\*]+?\b(axlbm_\w+)\s*\(", open({header!r}).read())))
calls = 0
for name in names:
    fn = getattr(L, name)
    if name == "axlbm_selftest_bounded_wait":  # launches a kernel whatever its arguments
        continue
    got = fn(*[t() for t in fn.argtypes])
    if name == "axlbm_abi_version":
        assert got == 5
    elif name == "axlbm_ws_weight_count":
        assert got > 0
    elif fn.restype is ctypes.c_char_p:
        assert got, name
    else:
        assert got == B.EINVAL, (name, got)
    calls += 1

# device layout of single domains
rng = np.random.default_rng(5)
layouts = 0
for _ in range(300):
    g = B.axlbm_grid(nr=int(rng.integers(-2, 5000)), nz=int(rng.integers(-2, 5000)),
                     precision=int(rng.integers(0, 5)), with_swirl=int(rng.integers(0, 3)),
                     with_temperature=int(rng.integers(0, 2)), collision=int(rng.integers(0, 3)), r0=0.0)
    n = ctypes.c_size_t()
    st = L.axlbm_state_bytes(ctypes.byref(g), ctypes.byref(n))
    assert st in (B.OK, B.EINVAL)
    if st == B.OK:
        planes = 9 + 4 * g.with_swirl + 4 * g.with_temperature
        assert n.value >= planes * g.nr * g.nz * {{0: 8, 1: 4}}.get(g.precision, 2)
        layouts += 1

# the batch planner
def planned(problems, precision):
    arr = B.domain_array(problems)
    n = ctypes.c_size_t()
    st = L.axlbm_batch_state_bytes(arr, len(problems), precision, ctypes.byref(n))
    assert st in (B.OK, B.EINVAL)
    if st == B.OK:
        planes = 17 if any(p.temperature for p in problems) else 13
        assert n.value >= planes * sum(p.nr * p.nz for p in problems) * (4 if precision == B.FP32 else 2)
    return st == B.OK

sweep = I.batch_sweep()
assert planned(sweep, B.FP32) and planned(sweep, B.FP16_DEV)
assert not planned([problem(8, 8, "pipe", swirl=False, temperature=False)], B.FP32)
assert not planned(sweep[:2], B.FP64)
mixes = sorted(BOUNDARY_MIXES)
batches = 0
for trial in range(150):
    doms = []
    for _ in range(int(rng.integers(1, 40))):
        nr = int(rng.choice([1, 2, 3, 17, 42, 43, 44, 127, 128, 129, 300]) if rng.random() < 0.5 else rng.integers(1, 260))
        nz = int(rng.integers(1, 260))
        mix = mixes[int(rng.integers(0, len(mixes)))]
        try:
            pb = problem(nr, nz, mix, temperature=bool(rng.integers(0, 2)))
        except (ValueError, AssertionError):
            continue
        if planned([pb], B.FP32):  # a domain a batch accepts on its own
            doms.append(pb)
    if doms:  # a list of such domains must always be packed
        assert planned(doms, B.FP32 if trial % 2 else B.FP16_DEV), [(p.nr, p.nz) for p in doms]
        batches += 1

# validation in axlbm_create (before any device work)
for change in (dict(tau=0.5), dict(r0=1.0), dict(z_lo="wall"), dict(rho0=-1.0)):
    kw = dict(nr=8, nz=8, tau=0.8)
    kw.update(change)
    pb = I.Problem(**kw)
    g, tau, f, b = B.structs(pb, "fp32")
    h = ctypes.c_void_p()
    st = L.axlbm_create(ctypes.byref(g), tau, ctypes.byref(f), ctypes.byref(b), None, None, 0, ctypes.byref(h))
    assert st == B.EINVAL and not h.value, change
print("calls", calls, "layouts", layouts, "batches", batches)
"""


def nvcc_or_skip():
    from paper_1003_0282_gb300 import build
    try:
        return build, build.nvcc()
    except RuntimeError:
        pytest.skip("no CUDA toolkit")


@pytest.fixture(scope="module")
def sanitized_lib(tmp_path_factory):
    build, cc = nvcc_or_skip()
    libasan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(libasan) or not os.path.exists(libasan):
        pytest.skip("gcc has no AddressSanitizer runtime here")
    out = tmp_path_factory.mktemp("abi_san")
    ptx_only = ["-gencode", "arch=compute_103a,code=compute_103a"]
    san = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined", "-Xcompiler",
           "-fno-sanitize-recover=undefined", "-Xcompiler", "-fno-omit-frame-pointer"]

    def compile_one(src):
        obj = str(out / (os.path.basename(src)[:-3] + ".o"))
        res = subprocess.run([cc, *ptx_only, *build.NVCC_FLAGS, *san, "-I", build.INCLUDE, "-c", src, "-o", obj],
                             capture_output=True, text=True)
        assert res.returncode == 0, res.stderr[-3000:]
        return obj

    srcs = build._sources()
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    lib = str(out / "libaxlbm_san.so")
    res = subprocess.run([cc, *ptx_only, "-shared", "-cudart", "static", *san, "-o", lib, *objs],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    return lib, libasan


def test_host_paths_are_clean_under_asan_and_ubsan(sanitized_lib):
    lib, libasan = sanitized_lib
    env = dict(os.environ, LD_PRELOAD=libasan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=0:exitcode=23",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1:exitcode=24", CUDA_VISIBLE_DEVICES="")
    script = DRIVER.format(root=ROOT, tests=TESTS, lib=lib, header=HEADER)
    out = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, timeout=900)
    report = out.stdout[-2000:] + out.stderr[-4000:]
    assert out.returncode == 0, report
    assert "runtime error" not in out.stderr and "AddressSanitizer" not in out.stderr, report
    words = out.stdout.split()
    counts = dict(zip(words[-6::2], map(int, words[-5::2])))
    assert counts["calls"] >= 50 and counts["layouts"] >= 50 and counts["batches"] >= 50, report
