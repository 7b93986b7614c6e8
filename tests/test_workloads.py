"""The batched workload's generator: 64 seeded problems within the stated
ranges (n, in-interval count, edge clusters, m0, n_c)."""
import numpy as np

from workloads import spectrum_config3


def test_config3_batch_ranges_and_determinism():
    ns, ms, ncs = [], [], set()
    for seed in range(64):
        lam, lmin, lmax, m0, n_c = spectrum_config3(seed)
        n = lam.size
        m = int(np.sum((lam > lmin) & (lam < lmax)))
        assert 512 <= n <= 4096 and 10 <= m <= 170
        assert m0 == int(np.ceil(1.5 * m)) and m0 < n
        assert n_c in (8, 16)
        ncs.add(n_c)
        # clustered edges: eigenvalues within 1e-3 of the half-width on both sides of each edge
        hw = 0.5 * (lmax - lmin)
        near = np.abs(lam - lmin) < 1e-3 * hw
        assert 2 <= np.sum(near | (np.abs(lam - lmax) < 1e-3 * hw)) <= 40
        assert np.all(np.diff(lam) >= 0)
        ns.append(n)
        ms.append(m)
        lam2, *_ = spectrum_config3(seed)
        np.testing.assert_array_equal(lam, lam2)
    assert ncs == {8, 16}
    assert min(ns) < 1500 and max(ns) > 3000   # the size range is exercised
    assert min(ms) < 50 and max(ms) > 120
