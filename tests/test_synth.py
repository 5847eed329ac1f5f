"""Seeded synthetic inputs: determinism, SU(3) links, Gaussian statistics."""

import numpy as np

import synth


def test_splitmix64_direct_indexing_matches_sequential_definition():
    """The n-th output equals the sequential SplitMix64 step applied n+1 times."""
    seed = 1234567
    mask = (1 << 64) - 1
    state = seed
    seq = []
    for _ in range(5):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        seq.append(z ^ (z >> 31))
    got = synth.splitmix64(seed, np.arange(5, dtype=np.uint64))
    assert [int(v) for v in got] == seq


def test_normals_statistics_and_chunking():
    z = synth.normals(5, 2_000_001)
    assert abs(z.mean()) < 5e-3 and abs(z.var() - 1) < 5e-3
    # any even starting offset reproduces the same stream
    assert np.array_equal(synth.normals(5, 1000, start=400), z[400:1400])


def test_gauge_links_are_special_unitary_and_reproducible():
    dims = (4, 4, 2, 2)
    U = synth.gauge_field(dims, 0.3, 1)
    assert U.shape == (64, 4, 3, 3)
    UdU = np.einsum("vmab,vmac->vmbc", U.conj(), U)
    assert np.abs(UdU - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    assert np.array_equal(U, synth.gauge_field(dims, 0.3, 1))
    assert not np.allclose(U, synth.gauge_field(dims, 0.3, 2))


def test_traceless_hermitian_generator_scale():
    """<tr H^2> = 8 for the traceless Hermitian part of a complex Gaussian matrix,
    so -i log U / eps recovers H with that mean."""
    eps = 0.05
    U = synth.gauge_field((8, 8, 8, 8), eps, 3).reshape(-1, 3, 3)[:4000]
    w = np.linalg.eigvals(U)
    h = np.angle(w) / eps
    assert abs((h ** 2).sum(axis=1).mean() - 8.0) < 0.3


def test_sources():
    dims = (4, 4, 4, 4)
    s = synth.gaussian_source(dims, 2)
    assert s.shape == (256, 4, 3) and abs(np.mean(np.abs(s) ** 2) - 2) < 0.2
    p = synth.point_source(dims, 2, 1)
    assert p[0, 2, 1] == 1 and np.count_nonzero(p) == 1


def test_uneven_batch_draws():
    b = synth.uneven_batch(16, 1)
    assert len(b) == 16
    assert all(d["dims"] in synth.UNEVEN_SHAPES for d in b)
    assert all(0.2 <= d["eps"] <= 0.35 and 0.11 <= d["kappa"] <= 0.124 for d in b)
    assert b == synth.uneven_batch(16, 1)
