"""Replaying runs of plain steps from captured CUDA graphs.

Every axlbm_step call ends with two check steps; the plain steps before them
run as whole (even, odd) pairs from graphs captured on first use.  The graph
path must give the populations and check values of launching every kernel,
bit for bit, for every boundary kind (its passes -- rings, axis mirror,
wet walls, Zou-He -- are nodes of the graph), in FP32 and FP64, from an even
or an odd level.
"""
import numpy as np
import pytest

from parity_util import BOUNDARY_MIXES, problem, seeded_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_0282_gb300 import build
    build.build()
    from paper_1003_0282_gb300 import axlbm
    return axlbm


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("mix", sorted(BOUNDARY_MIXES))
def test_single_domain_graphs_match_direct_launches(B, precision, mix):
    pb = problem(23, 17, mix, collision="mrt" if mix.startswith("nee") else "bgk")
    st = seeded_state(pb, seed=5)
    out = []
    for graphs in (True, False):
        dom = B.Domain(pb, precision)
        dom.use_graphs(graphs)
        dom.set_populations(st.f, st.g if pb.swirl else None, st.h if pb.temperature else None, time=0)
        dom.step(1)
        # too short for graphs; sizes the plain kernels; graph runs from an odd and an even level
        for n in (3, 21, 29, 30):
            dom.step(n)
        caps, launches = dom.graph_stats()
        assert (caps, launches > 0) == ((1, True) if graphs else (0, False)), (caps, launches)
        out.append((dom.get_populations(), dom.residual(), dom.time))
        dom.close()
    (p0, r0, t0), (p1, r1, t1) = out
    assert t0 == t1 == 84
    assert r0 == r1
    for x, y in zip(p0, p1):
        assert (x is None and y is None) or np.array_equal(x, y)
