"""The input generators: the batched workload's 64 seeded problems within the
stated ranges (n, in-interval count, edge clusters, m0, n_c), the disk
spectra and planted general matrices, the dense-edge stand-in spectrum."""
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


def test_disk_spectra_and_general_planted_matrices():
    from workloads import planted_general, spectrum_disk
    for real in (False, True):
        c = 0.4 if real else 0.4 - 0.2j
        lam = spectrum_disk(3, 60, 12, center=c, radius=2.0, gap=0.1, outer=5.0, real_pairs=real)
        d = np.abs(lam - c)
        assert lam.size == 60 and np.sum(d < 2.0) == 12
        assert np.all((d < 2.0 * 0.9) | ((d > 2.0 * 1.1) & (d < 10.0)))
        if real:
            np.testing.assert_allclose(lam[30:], np.conj(lam[:30]), rtol=0, atol=0)
        A, V = planted_general(lam, 5, cond=6.0, real=real)
        assert A.dtype == (np.float64 if real else np.complex128)
        # the planted pairs are eigenpairs and the eigenvector basis is as conditioned as stated
        assert np.max(np.abs(A @ V - V * lam[None, :])) < 1e-11 * np.linalg.norm(A, 2)
        if not real:
            assert np.linalg.cond(V) <= 6.0 * (1 + 1e-9)
        np.testing.assert_array_equal(spectrum_disk(3, 60, 12, center=c, radius=2.0, gap=0.1, outer=5.0,
                                                    real_pairs=real), lam)


def test_dense_edge_spectrum():
    from workloads import spectrum_dense_edge
    lam, a, b = spectrum_dense_edge(0)
    assert lam.size == 600 and np.all(np.diff(lam) > 0)
    assert np.sum((lam > a) & (lam < b)) == 43
    # the group straddles the upper edge: 15 inside and 15 outside within 0.05
    near = lam[np.abs(lam - b) < 0.05]
    assert np.sum(near < b) == 15 and np.sum(near > b) == 15
    assert np.min(np.abs(lam - b)) > 1e-4
    np.testing.assert_array_equal(lam, spectrum_dense_edge(0)[0])
