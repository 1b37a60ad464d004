"""Pins of the oracle's metal-trace estimation (Sec. "Real metal artifacts"): the disk
dilation against scipy.ndimage with the same structuring element, and the trace against
the union of the brute-force supports of the marked pixels' columns of R_h."""
import numpy as np
import pytest
import scipy.ndimage

import oracle
from oracle import Geometry


@pytest.mark.parametrize("radius", [0, 1, 2, 5])
def test_dilation_matches_scipy(radius):
    rng = np.random.default_rng(radius)
    m = rng.uniform(size=(23, 19)) > 0.97
    yy, xx = np.mgrid[-radius:radius + 1, -radius:radius + 1]
    disk = (yy * yy + xx * xx) <= radius * radius
    ref = scipy.ndimage.binary_dilation(m, structure=disk)
    np.testing.assert_array_equal(oracle.dilate_disk(m, radius), ref)


def test_trace_is_the_union_of_supports():
    """A bin is in the trace iff the marked pixels' brute-force R_h entries there (the
    hat-weight formulation, not the projector) sum above the tolerance."""
    n, N, M = 12, 9, 17
    geo = Geometry(n, N, M)
    u = np.zeros((n, n))
    u[4, 7] = 5.0
    u[8, 2] = 4.0
    marked, trace = oracle.metal_trace_estimate(u, geo, 1.0, radius=1)
    assert marked.sum() == 2 * 5
    ls, ks = np.meshgrid(np.arange(N), np.arange(M), indexing="ij")
    ls, ks = ls.ravel(), ks.ravel()
    acc = np.zeros(N * M)
    for i, j in zip(*np.nonzero(marked)):
        e = np.zeros((n, n))
        e[i, j] = 1.0
        acc += oracle.rh_forward_entries(e, geo, ls, ks)
    np.testing.assert_array_equal(trace.ravel().astype(bool), acc > 1e-6)
    assert 0 < trace.sum() < N * M
