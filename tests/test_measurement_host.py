"""Host-side pieces of the measurement tools (no GPU): the HEALPix ring table that the
ring-FFT / cuFFT comparison groups rings by."""
import numpy as np

import synthetic as S
from profile_step import ring_table


def test_ring_table_tiles_the_sphere_ring_by_ring():
    for N in (1, 2, 8, 32):
        t = ring_table(N)
        assert len(t) == 4 * N - 1
        assert t[0] == (0, 4)
        assert sum(n for _, n in t) == 12 * N * N
        assert all(t[k][0] + t[k][1] == t[k + 1][0] for k in range(len(t) - 1))
        # ring lengths 4i in the caps, 4N in the belt, mirrored north/south
        assert [n for _, n in t] == [n for _, n in reversed(t)]
        z, _ = S.pixel_positions(N)
        for first, n in t:
            assert np.ptp(z[first:first + n]) < 1e-12   # one ring = one latitude
        zr = [z[f] for f, _ in t]
        assert all(a > b for a, b in zip(zr, zr[1:]))    # north to south
