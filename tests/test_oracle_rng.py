"""Pins of the oracle's random numbers: Philox4x64-10 and Marsaglia's sphere sampler."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("key", [(0, 0), (1, 2), (0xDEADBEEF12345678, 7), (2**64 - 1, 2**63)])
@pytest.mark.parametrize("ctr", [(0, 0, 0, 0), (5, 9, 3, 2), (2**64 - 2, 1, 2**40, 3)])
def test_philox_matches_numpy(key, ctr):
    # numpy's Philox bit generator (a library implementation of Philox4x64-10) advances its
    # counter by one before the first block, so block n of a generator started at counter c
    # is Philox(c + 1 + n); the carry propagates into the higher words.
    bg = np.random.Philox(key=np.array(key, np.uint64), counter=np.array(ctr, np.uint64))
    got = bg.random_raw(8)
    base = int(ctr[0]) + (int(ctr[1]) << 64) + (int(ctr[2]) << 128) + (int(ctr[3]) << 192)
    for n in range(2):
        c = base + 1 + n
        words = [(c >> (64 * q)) & (2**64 - 1) for q in range(4)]
        ours = O.philox(words, key)
        assert list(ours) == list(got[4 * n:4 * n + 4])


def _sample_sphere(n, seed=3):
    out = []
    c = 0
    while len(out) < n:
        w = O.philox((c, 0, 0, O.TAG_INIT), (seed, 0))
        c += 1
        s = O.marsaglia(w[0], w[1])
        if s is not None:
            out.append(s)
    return np.array(out), c


def test_marsaglia_unit_norm_and_moments():
    S, tries = _sample_sphere(40000)
    n = len(S)
    assert np.all(np.abs(np.linalg.norm(S, axis=1) - 1.0) < 4e-16)
    # acceptance of the disc test is pi/4
    acc = n / tries
    assert abs(acc - np.pi / 4) < 5 * np.sqrt(acc * (1 - acc) / tries)
    # uniform on the sphere: <S_a> = 0 (var 1/3), <S_a S_b> = delta_ab / 3
    mean = S.mean(0)
    assert np.all(np.abs(mean) < 5 * np.sqrt(1 / 3 / n))
    M = S.T @ S / n
    assert np.allclose(np.diag(M), 1 / 3, atol=5 * np.sqrt(4 / 45 / n))
    off = M[np.triu_indices(3, 1)]
    assert np.all(np.abs(off) < 5 * np.sqrt(1 / 15 / n))
    # Archimedes: S_z is uniform on [-1, 1]
    hist, _ = np.histogram(S[:, 2], bins=20, range=(-1, 1))
    exp = n / 20
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 50  # 19 dof, p ~ 1e-4


def test_marsaglia_rejects_outside_disc():
    # words giving a1 = a2 = 0 (s == 0) and a1 = -1 (s >= 1) are rejected
    half = 1 << 63  # u = 1/2 -> a = 0
    assert O.marsaglia(half, half) is None
    assert O.marsaglia(0, half) is None
    S = O.marsaglia(half + (1 << 61), half)  # u = 0.625 -> a1 = 0.25, a2 = 0
    assert S is not None
    s = 0.0625
    assert S[0] == 2 * 0.25 * np.sqrt(1 - s) and S[1] == 0.0 and S[2] == 1 - 2 * s
