"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer.

The oracle's C source is built with -fsanitize=address,undefined into a
temporary library, and every entry point runs in a subprocess with the ASan
runtime preloaded:
- every boundary mix;
- both collision models, with and without the g and h distributions;
- grids from the smallest each mix accepts up to several nodes per side.

An out-of-bounds access, a use of freed memory, a signed overflow, a
misaligned or null access or any other undefined behaviour makes the
subprocess print a report and exit non-zero, which fails the test.  Nothing
here touches the GPU or the CUDA library.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(ROOT, "oracle", "axlbm_oracle.c")

DRIVER = r"""
import sys
import numpy as np
sys.path[:0] = [{root!r}, {tests!r}]
import oracle
from parity_util import BOUNDARY_MIXES, problem, seeded_state

cases = 0
for mix in sorted(BOUNDARY_MIXES):
    for collision in ("bgk", "mrt"):
        for swirl, temperature in ((True, True), (True, False), (False, False)):
            for nr, nz in ((1, 1), (2, 1), (1, 3), (2, 2), (3, 3), (6, 5)):
                try:
                    pb = problem(nr, nz, mix, swirl=swirl, temperature=temperature, collision=collision)
                except (ValueError, AssertionError):
                    continue
                if not oracle.validate(pb):
                    continue
                st = seeded_state(pb, seed=nr * 10 + nz)
                oracle.step(st, 3)
                oracle.moments(st)
                oracle.stats(st)
                fn, gn, hn = oracle.stream(pb, st.f, st.g, st.h)
                assert np.all(np.isfinite(fn)), (mix, nr, nz)
                for r in oracle.node_radii(pb)[:2]:
                    oracle.collide_cell(pb, r, 1e-6, st.f[:, 0, 0], st.g[:, 0, 0], st.h[:, 0, 0])
                cases += 1
oracle.mrt_matrix()
print("cases", cases)
"""


def run_sanitized(tmp_path, source):
    """Build `source` (oracle C text) with ASan and UBSan and run the DRIVER script on it."""
    libasan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(libasan) or not os.path.exists(libasan):
        pytest.skip("gcc has no AddressSanitizer runtime here")
    src = tmp_path / "axlbm_oracle.c"
    src.write_text(source)
    lib = tmp_path / "liboracle_san.so"
    subprocess.run(["gcc", "-O1", "-g", "-std=c11", "-fPIC", "-shared", "-Wall", "-fno-omit-frame-pointer",
                    "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-o", str(lib), str(src),
                    "-lm"], check=True)
    env = dict(os.environ, LD_PRELOAD=libasan, AXLBM_ORACLE_LIB=str(lib),
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=0:exitcode=23",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1:exitcode=24")
    return subprocess.run([sys.executable, "-c", DRIVER.format(root=ROOT, tests=TESTS)], env=env,
                          capture_output=True, text=True, timeout=600)


def test_oracle_is_clean_under_asan_and_ubsan(tmp_path):
    out = run_sanitized(tmp_path, open(SRC).read())
    report = out.stdout[-2000:] + out.stderr[-4000:]
    assert out.returncode == 0, report
    assert "runtime error" not in out.stderr and "AddressSanitizer" not in out.stderr, report
    cases = int(out.stdout.split("cases")[-1])
    assert cases >= 13 * 2 * 3 * 3, report  # every mix, model and distribution set on several grids


def test_the_harness_catches_a_planted_overflow(tmp_path):
    """One read past the end of f in the moments loop must end the run with an ASan report."""
    text = open(SRC).read()
    good = "for (int a = 0; a < 9; ++a) fi[a] = f[a * n + x];"
    assert text.count(good) >= 1
    out = run_sanitized(tmp_path, text.replace(good, "for (int a = 0; a < 10; ++a) fi[a % 9] = f[a * n + x];", 1))
    assert out.returncode == 23 and "heap-buffer-overflow" in out.stderr, out.stderr[-2000:]
