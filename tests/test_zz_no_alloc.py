"""axlbm_check_static: the check-step statistics for callers that cannot allocate.

Some callers cannot call cudaMalloc (code inside another framework's memory
pool, or a loop that forbids allocations after start-up); this entry point
gives them the check-step reduction with its scratch in a fixed device array.
The test compares it, through the C ABI, with what the regular check step of
axlbm_step reports, on two calls in a row: the first without and the second
with the previous level's speeds; on the half-spacing grid, with a node on
the axis, with an inner wall at r0 > 0, and with wet walls.  The test
allocates its own buffers (it is the caller); the entry point allocates
nothing.
"""
import math

import numpy as np
import pytest

from parity_util import problem, seeded_state, upload

pytestmark = pytest.mark.gpu


# the inner kinds whose radius differs (half-spacing axis, node on the axis,
# an inner wall at r0 > 0) and a domain with wet walls on three faces
CASES = [("crystal", 150, 37), ("axis-node-crystal", 150, 37), ("annulus-mixed", 133, 29), ("nee-axis-node", 97, 23)]


@pytest.mark.parametrize("mix,nr,nz", CASES)
def test_check_static_matches_the_check_step(mix, nr, nz):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_0282_gb300 import build
    build.build()
    from paper_1003_0282_gb300 import axlbm as B

    pb = problem(nr, nz, mix)   # swirl and temperature on, a few tiles with ragged tails
    dom = B.Domain(pb, "fp64")
    upload(dom, seeded_state(pb, 31))
    k = 9
    dom.step(k - 1)
    f1, g1, h1 = dom.get_populations()      # level k - 1
    dom.step(1)                             # checks level k - 1
    _, mass1, budget1 = dom.residual()
    f2, g2, h2 = dom.get_populations()      # level k
    dom.step(1)                             # checks level k against k - 1
    res2, mass2, budget2 = dom.residual()
    dom.close()

    grid, tau, forcing, bc = B.structs(pb, "fp64")
    n = pb.nr * pb.nz
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    speed1 = torch.empty(n, dtype=torch.float64, device="cuda")
    out1 = torch.full((4,), math.nan, dtype=torch.float64, device="cuda")
    out2 = torch.full((4,), math.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    a_z = lambda t: pb.az0 * math.cos(pb.omega_t * t)
    d1 = [dev(f1), dev(g1), dev(h1)]
    d2 = [dev(f2), dev(g2), dev(h2)]
    B.axlbm_check_static(grid, tau, forcing, bc, d1[0].data_ptr(), d1[1].data_ptr(), d1[2].data_ptr(),
                         a_z(k - 1), 0, speed1.data_ptr(), out1.data_ptr(), stream)
    B.axlbm_check_static(grid, tau, forcing, bc, d2[0].data_ptr(), d2[1].data_ptr(), d2[2].data_ptr(), a_z(k),
                         speed1.data_ptr(), 0, out2.data_ptr(), stream)
    torch.cuda.synchronize()
    o1, o2 = out1.cpu().numpy(), out2.cpu().numpy()
    assert o1[0] == 0.0 and o1[3] == 0.0 and o2[3] == 0.0
    assert o1[1] == pytest.approx(mass1, rel=1e-12)
    assert o1[2] == pytest.approx(budget1, rel=1e-9, abs=1e-15)
    assert o2[1] == pytest.approx(mass2, rel=1e-12)
    assert o2[2] == pytest.approx(budget2, rel=1e-9, abs=1e-15)
    assert o2[0] == pytest.approx(res2, rel=1e-9, abs=1e-15)


def test_check_static_rejects_an_axis_off_zero_and_unknown_inner_kinds():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_0282_gb300 import axlbm as B

    pb = problem(16, 8, "axis-node-pipe")
    grid, tau, forcing, bc = B.structs(pb, "fp64")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    f = torch.zeros(17 * 16 * 8, dtype=torch.float64, device="cuda")  # never read: the checks come first
    grid.r0 = 1.0
    with pytest.raises(B.AxlbmError) as ei:
        B.axlbm_check_static(grid, tau, forcing, bc, f.data_ptr(), f.data_ptr(), f.data_ptr(), 0.0, 0, 0,
                             out.data_ptr(), 0)
    assert ei.value.status == B.EINVAL
    grid.r0 = 0.0
    bc.inner = 7
    with pytest.raises(B.AxlbmError) as ei:
        B.axlbm_check_static(grid, tau, forcing, bc, f.data_ptr(), f.data_ptr(), f.data_ptr(), 0.0, 0, 0,
                             out.data_ptr(), 0)
    assert ei.value.status == B.EINVAL


def test_check_static_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_0282_gb300 import axlbm as B
    from paper_1003_0282_gb300 import inputs as I

    grid, tau, forcing, _ = B.structs(I.Problem(nr=4096, nz=1025, tau=0.8), "fp64")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    f = torch.zeros(16, dtype=torch.float64, device="cuda")  # never read: the size check comes first
    with pytest.raises(B.AxlbmError) as ei:
        B.axlbm_check_static(grid, tau, forcing, None, f.data_ptr(), 0, 0, 0.0, 0, 0, out.data_ptr(), 0)
    assert ei.value.status == B.EINVAL
    assert "4,194,304" in B.lib().axlbm_last_error(None).decode()
