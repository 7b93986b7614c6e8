"""Planted-spectrum test matrices and seeded starting subspaces.

A planted problem is A = Q diag(lambda) Q^H with Q drawn from the QR
factorisation of a seeded Gaussian matrix, so the eigenpairs inside the search
interval (lambda_min, lambda_max) are known in closed form.  The spectra follow
the workloads of the paper (Sect. III: n = 545, 50 eigenvalues in [-1, 1], the
other 495 either spread over [1.01, 20.81] or packed in [1.01, 1.1]) and the
larger edge-clustered workloads the eigensolver is benchmarked on.

Everything here is input generation: no quadrature, no factorisation, no
Rayleigh-Ritz.  All arrays are returned in column-major (Fortran) order, the
layout the C interface expects.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Planted eigenvalues keep at least this distance from an interval edge, so an
# open interval test on them is never decided by rounding.
EDGE_MARGIN = 1e-12


@dataclass
class Problem:
    """One planted Hermitian (or real symmetric) eigenproblem."""

    name: str
    A: np.ndarray            # n x n, Fortran order, float64 or complex128
    lam: np.ndarray          # all n planted eigenvalues, ascending
    Q: np.ndarray | None     # n x n eigenvectors (columns match lam), or None
    lmin: float
    lmax: float
    m0: int
    n_c: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.shape[0]

    @property
    def is_complex(self) -> bool:
        return np.iscomplexobj(self.A)

    @property
    def inside(self) -> np.ndarray:
        """Planted eigenvalues strictly inside (lmin, lmax), ascending."""
        return self.lam[(self.lam > self.lmin) & (self.lam < self.lmax)]

    @property
    def inside_vectors(self) -> np.ndarray:
        mask = (self.lam > self.lmin) & (self.lam < self.lmax)
        return self.Q[:, mask]

    @property
    def anorm(self) -> float:
        """Exact spectral norm max |lambda| of the planted matrix."""
        return float(np.max(np.abs(self.lam)))


def _uniform_avoiding(rng, count, lo, hi, lmin, lmax, gap):
    """`count` draws uniform on [lo, lmin - gap) U (lmax + gap, hi]."""
    left = max(0.0, (lmin - gap) - lo)
    right = max(0.0, hi - (lmax + gap))
    total = left + right
    u = rng.uniform(0.0, total, size=count)
    out = np.where(u < left, lo + u, (lmax + gap) + (u - left))
    return out


def spectrum_edge_clusters(rng, n, m_in, lmin, lmax, bulk_lo, bulk_hi,
                           n_edge_in=0, n_edge_out=0, width=0.0):
    """Eigenvalues with clusters hugging both interval edges.

    m_in eigenvalues lie strictly inside (lmin, lmax); n_edge_in of them per
    edge sit within `width` inside that edge.  n_edge_out per edge sit within
    `width` outside it.  The rest of the n eigenvalues are uniform on
    [bulk_lo, bulk_hi] outside the interval (and outside the edge bands when
    there are outside clusters).
    """
    assert 2 * n_edge_in <= m_in
    n_out_bulk = n - m_in - 2 * n_edge_out
    assert n_out_bulk >= 0
    parts = []
    if n_edge_in:
        parts.append(lmin + rng.uniform(EDGE_MARGIN, width, n_edge_in))
        parts.append(lmax - rng.uniform(EDGE_MARGIN, width, n_edge_in))
    inner = m_in - 2 * n_edge_in
    lo_in = lmin + (width if n_edge_in else EDGE_MARGIN)
    hi_in = lmax - (width if n_edge_in else EDGE_MARGIN)
    parts.append(rng.uniform(lo_in, hi_in, inner))
    if n_edge_out:
        parts.append(lmin - rng.uniform(EDGE_MARGIN, width, n_edge_out))
        parts.append(lmax + rng.uniform(EDGE_MARGIN, width, n_edge_out))
    gap = width if n_edge_out else EDGE_MARGIN
    parts.append(_uniform_avoiding(rng, n_out_bulk, bulk_lo, bulk_hi, lmin, lmax, gap))
    lam = np.sort(np.concatenate(parts))
    assert lam.size == n
    assert np.sum((lam > lmin) & (lam < lmax)) == m_in
    return lam


def spectrum_config1(seed=0):
    """n = 500 real symmetric: 40 of 500 eigenvalues in I = [-1, 1], 5 of them
    within 1e-3 of each edge; the other 460 uniform in [-10, 10] outside I."""
    rng = np.random.default_rng(seed)
    lam = spectrum_edge_clusters(rng, 500, 40, -1.0, 1.0, -10.0, 10.0,
                                 n_edge_in=5, n_edge_out=0, width=1e-3)
    return lam, -1.0, 1.0


def spectrum_config2(seed=0, n=8192, m_in=200, edge_in=30, edge_out=60,
                     width=1e-4, bulk=50.0):
    """Complex Hermitian edge-clustered spectrum: m_in eigenvalues in [-1, 1]
    with edge_in packed within `width` inside each edge, edge_out packed within
    `width` outside each edge, the rest uniform in [-bulk, bulk] outside I.
    Defaults are the n = 8192 single-large-problem workload."""
    rng = np.random.default_rng(seed)
    lam = spectrum_edge_clusters(rng, n, m_in, -1.0, 1.0, -bulk, bulk,
                                 n_edge_in=edge_in, n_edge_out=edge_out, width=width)
    return lam, -1.0, 1.0


def spectrum_config3(seed, scale=1.0):
    """One problem of the batched workload (64 independent real symmetric
    problems, seeds 0..63): n uniform in 512..4096, m uniform in 10..170
    eigenvalues inside the problem's own interval, an edge cluster of 2..20
    eigenvalues per edge within 1e-3 of it, half of each cluster inside and half
    outside (the reading of the unspecified cluster side), the rest uniform
    over an outer range 10x the interval's half-width; m0 = ceil(1.5 m),
    n_c = 8 or 16.  Returns (lam, lmin, lmax, m0, n_c)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 3]))
    n = int(rng.integers(512, 4097))
    m = int(rng.integers(10, 171))
    if scale != 1.0:    # the same draw scaled down (small parity cases)
        n = max(64, int(n * scale))
        m = max(4, int(m * scale))
    cl = int(rng.integers(2, 21))
    c_in = min(cl // 2, m // 2)
    c_out = cl - cl // 2
    if scale != 1.0:
        cl = max(2, int(cl * scale))
        c_in = min(cl // 2, m // 2)
        c_out = cl - cl // 2
    c = float(rng.uniform(-5.0, 5.0))
    r = float(rng.uniform(0.5, 2.0))
    lmin, lmax = c - r, c + r
    lam = spectrum_edge_clusters(rng, n, m, lmin, lmax, c - 10.0 * r, c + 10.0 * r,
                                 n_edge_in=c_in, n_edge_out=c_out, width=1e-3 * r)
    m0 = int(np.ceil(1.5 * m))
    n_c = int(rng.choice([8, 16]))
    return lam, lmin, lmax, m0, n_c


def spectrum_config4(seed, n=2048):
    """One spectrum of the learned-proposer workload (2000 training and 500
    held-out real symmetric problems, seeds 0..1999 and 10000..10499): n = 2048
    eigenvalues, I = [-1, 1], m uniform in 10..170 eigenvalues inside, an edge
    cluster at each edge of c eigenvalues (c uniform in 0..40; half inside and
    half outside the edge, the reading of the unspecified side) within a
    width w log-uniform in [1e-6, 1e-1], the rest uniform in [-10, 10] outside
    I and outside the edge bands.  Returns (lam, lmin, lmax, meta)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 4]))
    m = int(rng.integers(10, 171))
    c = int(rng.integers(0, 41))
    w = float(10.0 ** rng.uniform(-6.0, -1.0))
    c_in = min(c // 2, m // 2)
    c_out = c - c // 2
    lam = spectrum_edge_clusters(rng, n, m, -1.0, 1.0, -10.0, 10.0, n_edge_in=c_in, n_edge_out=c_out, width=w)
    return lam, -1.0, 1.0, {"m": m, "cluster": c, "width": w, "edge_in": c_in, "edge_out": c_out}


def spectrum_config5(seed=0, n=32768, m_in=700, edge_out=80, width=1e-5, bulk=50.0):
    """The largest single problem: real symmetric n = 32768, 700 eigenvalues
    uniform in I = [-1, 1], 80 packed within 1e-5 outside each edge (the
    hard case of Sect. I: eigenvalues just outside the interval), the rest
    uniform in [-50, 50] outside I and the edge bands (m0 = 1000, n_c = 8
    upper-half nodes)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 5]))
    lam = spectrum_edge_clusters(rng, n, m_in, -1.0, 1.0, -bulk, bulk, n_edge_in=0, n_edge_out=edge_out,
                                 width=width)
    return lam, -1.0, 1.0


def spectrum_paper(kind, seed=0, n=545, m_in=50):
    """The two n = 545 spectra of the paper's Sect. III experiments: 50
    eigenvalues in I = [-1, 1]; the other 495 in [1.01, 20.81] ("Sparse") or
    [1.01, 1.1] ("Dense").  The in-interval eigenvalues are drawn uniformly."""
    rng = np.random.default_rng(seed)
    hi = {"sparse": 20.81, "dense": 1.1}[kind]
    inside = rng.uniform(-1.0 + EDGE_MARGIN, 1.0 - EDGE_MARGIN, m_in)
    outside = rng.uniform(1.01, hi, n - m_in)
    return np.sort(np.concatenate([inside, outside])), -1.0, 1.0


def spectrum_dense_edge(seed=0, n=600, m_in=43, group=30, width=0.1, bulk=20.0):
    """A stand-in for the second interval of the paper's Fig. 4 (43 pairs,
    its upper edge through the middle of a dense group of eigenvalues; the
    Hamiltonian itself is not available): I = [-1, 1] holds m_in eigenvalues,
    group of them equally spaced across (1 - width/2, 1 + width/2), half
    inside and half outside, the other inside ones uniform in
    (-0.95, 1 - width/2), the rest uniform in [-bulk, -1.1] and [1.2, bulk]."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 7]))
    g_in, g_out = group // 2, group - group // 2
    half = width / 2
    grp_in = 1.0 - half + (np.arange(g_in) + 0.5) * half / g_in
    grp_out = 1.0 + (np.arange(g_out) + 0.5) * half / g_out
    rest_in = rng.uniform(-0.95, 1.0 - half, m_in - g_in)
    n_out = n - m_in - g_out
    lo = rng.uniform(-bulk, -1.1, n_out // 2)
    hi = rng.uniform(1.2, bulk, n_out - n_out // 2)
    return np.sort(np.concatenate([rest_in, grp_in, grp_out, lo, hi])), -1.0, 1.0


def spectrum_uniform(n, m_in, seed=0, lmin=-1.0, lmax=1.0, bulk=10.0):
    """Uniform spectrum with exactly m_in eigenvalues in (lmin, lmax)."""
    rng = np.random.default_rng(seed)
    lam = spectrum_edge_clusters(rng, n, m_in, lmin, lmax, lmin - bulk, lmax + bulk)
    return lam, lmin, lmax


def haar_unitary(n, seed, complex_=False):
    """Q from the Householder QR of a seeded N(0,1) (or complex Gaussian)
    matrix, with the phases of diag(R) absorbed so Q is Haar distributed."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    if complex_:
        G = (G + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    Qm, R = np.linalg.qr(G)
    d = np.diag(R)
    ph = d / np.abs(d)
    return np.asfortranarray(Qm * ph[None, :])


def planted_matrix(Q, lam):
    """A = Q diag(lam) Q^H, made exactly Hermitian, Fortran order."""
    A = (Q * lam[None, :]) @ Q.conj().T
    A = 0.5 * (A + A.conj().T)
    return np.asfortranarray(A)


def planted_pencil(lam, seed, complex_=False, cond=10.0):
    """A planted generalized problem A x = lambda B x: B = L L^H with L lower
    triangular (seeded, diagonal in [1, cond]), Q Haar, A = L Q diag(lam) Q^H
    L^H, so the eigenvalues are lam and the B-orthonormal eigenvectors are
    X = L^{-H} Q.  Returns (A, B, X), Fortran order."""
    n = lam.size
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xB]))
    Lm = np.tril(rng.standard_normal((n, n)), -1) / np.sqrt(n)
    if complex_:
        Lm = Lm + 1j * np.tril(rng.standard_normal((n, n)), -1) / np.sqrt(n)
    Lm = Lm + np.diag(rng.uniform(1.0, cond, n))
    Q = haar_unitary(n, seed + 2000, complex_)
    LQ = Lm @ Q
    A = (LQ * lam[None, :]) @ LQ.conj().T
    B = Lm @ Lm.conj().T
    X = np.linalg.solve(Lm.conj().T, Q)
    return (np.asfortranarray(0.5 * (A + A.conj().T)), np.asfortranarray(0.5 * (B + B.conj().T)),
            np.asfortranarray(X))


def spectrum_disk(seed, n, m_in, center=0.0 + 0.0j, radius=1.0, gap=0.1, outer=10.0, real_pairs=False):
    """Complex eigenvalues for the general (non-Hermitian) problem: m_in
    uniform in the disk |z - center| < radius (1 - gap), the other n - m_in
    uniform in the annulus radius (1 + gap) < |z - center| < outer radius.
    real_pairs: the spectrum of a real matrix (closed under conjugation,
    center real, n and m_in even)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xD15C]))

    def disk(count, r0, r1):
        rho = np.sqrt(rng.uniform(r0 * r0, r1 * r1, count))
        return rho * np.exp(2j * np.pi * rng.uniform(0.0, 1.0, count))

    if real_pairs:
        if n % 2 or m_in % 2 or complex(center).imag != 0.0:
            raise ValueError("real_pairs needs even n, m_in and a real center")
        a = disk(m_in // 2, 0.0, radius * (1.0 - gap))
        b = disk((n - m_in) // 2, radius * (1.0 + gap), outer * radius)
        half = np.concatenate([a, b])
        lam = np.concatenate([half, np.conj(half)])
    else:
        lam = np.concatenate([disk(m_in, 0.0, radius * (1.0 - gap)), disk(n - m_in, radius * (1.0 + gap),
                                                                          outer * radius)])
    return center + lam


def planted_general(lam, seed, cond=10.0, real=False):
    """A general (non-normal) matrix with eigenvalues lam: A = V diag(lam)
    V^{-1} with V = Q1 diag(s) Q2, Q1 and Q2 Haar unitary and singular values
    s log-uniform in [1, cond] (eigenvector condition number <= cond).  real:
    lam closed under conjugation and listed as (half, conj(half)); then V keeps
    the first half of those columns and appends their conjugates, so A is real
    (that V's conditioning is no longer bounded by cond).  Returns (A, V),
    Fortran order."""
    lam = np.asarray(lam, dtype=np.complex128)
    n = lam.size
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x6E4]))
    s = np.exp(rng.uniform(0.0, np.log(cond), n))
    Q1 = haar_unitary(n, seed + 3000, True)
    Q2 = haar_unitary(n, seed + 4000, True)
    V = (Q1 * s[None, :]) @ Q2
    if real:
        h = n // 2
        if not np.allclose(lam[h:], np.conj(lam[:h])):
            raise ValueError("real: lam must be (half, conj(half))")
        V = np.concatenate([V[:, :h], np.conj(V[:, :h])], axis=1)
    Vinv = np.linalg.inv(V)
    A = (V * lam[None, :]) @ Vinv
    if real:
        A = A.real
    return np.asfortranarray(A), np.asfortranarray(V)


def random_subspace(n, m, seed, complex_=False):
    """Seeded N(0,1) starting subspace X0 (n x m), Fortran order.  Complex
    entries have independent N(0, 1/2) real and imaginary parts."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5EED]))
    X = rng.standard_normal((n, m))
    if complex_:
        X = (X + 1j * rng.standard_normal((n, m))) / np.sqrt(2.0)
    return np.asfortranarray(X)


def make_problem(name, lam, lmin, lmax, m0, n_c, seed=0, complex_=False, keep_q=True):
    Q = haar_unitary(lam.size, seed + 1000, complex_)
    A = planted_matrix(Q, lam)
    return Problem(name=name, A=A, lam=lam, Q=Q if keep_q else None,
                   lmin=lmin, lmax=lmax, m0=m0, n_c=n_c,
                   meta={"seed": seed, "complex": complex_})


def gaussian_torch(n, seed, complex_=False, gen="torch_cpu"):
    """The seeded Gaussian whose QR gives Q for the large planted matrices:
    gen "torch_cpu" draws it with torch's CPU generator (reproducible on any
    host), "numpy" with numpy's (the draw of haar_unitary), "torch_cuda" with
    the CUDA generator on the current GPU (not reproducible on a host)."""
    import torch

    dt = torch.complex128 if complex_ else torch.float64
    if gen == "numpy":
        rng = np.random.default_rng(int(seed))
        G = rng.standard_normal((n, n))
        if complex_:
            G = (G + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
        return torch.from_numpy(G)
    dev = "cuda" if gen == "torch_cuda" else "cpu"
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed))
    return torch.randn((n, n), generator=g, dtype=dt, device=dev)


def planted_matrix_torch(lam, seed, complex_=False, device="cuda:0", gen="torch_cpu"):
    """A = Q diag(lam) Q^H with Q from the QR factorisation (on the GPU) of the
    seeded Gaussian gaussian_torch(n, seed + 1000, gen).  Returns the
    column-major CUDA tensor A; Q is not kept."""
    import torch

    n = int(lam.size)
    dt = torch.complex128 if complex_ else torch.float64
    G = gaussian_torch(n, int(seed) + 1000, complex_, gen).to(device=device, dtype=dt)
    Q, R = torch.linalg.qr(G)
    d = torch.diagonal(R)
    Q = Q * (d / d.abs())[None, :]
    del G, R
    lam_t = torch.as_tensor(lam, dtype=torch.float64, device=device).to(dt)
    A = (Q * lam_t[None, :]) @ Q.conj().T
    del Q
    A = 0.5 * (A + A.conj().T)
    return A.transpose(0, 1).contiguous().transpose(0, 1)


def planted_block_host(lam, seed, rows, complex_=False, gen="torch_cpu"):
    """The leading rows x rows block of the matrix planted_matrix_torch builds
    with a host-reproducible generator (same spectrum and Gaussian; Q from the
    host's QR, equal up to rounding): Q[:rows] diag(lam) Q[:rows]^H."""
    import torch

    G = gaussian_torch(lam.size, int(seed) + 1000, complex_, gen)
    Q, R = torch.linalg.qr(G)
    d = torch.diagonal(R)
    Q = (Q * (d / d.abs())[None, :])[:rows].numpy()
    B = (Q * lam[None, :]) @ Q.conj().T
    return np.asfortranarray(0.5 * (B + B.conj().T))
