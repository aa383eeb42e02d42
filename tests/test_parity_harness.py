"""The windowed oracle used for full-size sampled parity is exact.

Advancing a window of half-width s around a node by s steps must give the
same populations at the node as advancing the whole domain (CPU only)."""
import numpy as np
import pytest

import oracle
from parity_util import BOUNDARY_MIXES, problem, seeded_state, window_oracle


@pytest.mark.parametrize("mix", sorted(BOUNDARY_MIXES))
def test_window_equals_full_domain(mix):
    pb = problem(23, 17, mix)
    st = seeded_state(pb, 5)
    pops = (st.f.copy(), st.g.copy(), st.h.copy())
    full = st.copy()
    oracle.step(full, 3)
    for (j, k) in [(0, 0), (0, 16), (22, 0), (22, 16), (11, 8), (1, 1), (21, 15), (5, 16), (0, 8), (11, 0)]:
        f, g, h = window_oracle(pops, pb, j, k, 3, 0)
        assert np.array_equal(f, full.f[:, k, j])
        if pb.swirl:
            assert np.array_equal(g, full.g[:, k, j])
        if pb.temperature:
            assert np.array_equal(h, full.h[:, k, j])
