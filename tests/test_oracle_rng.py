"""Pins for the counter-based Rademacher generator (oracle side)."""
import os

import numpy as np

from oracle import rng

GOLD = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")


def test_splitmix64_known_answer():
    want = [int(l) for l in open(GOLD) if l.strip() and not l.startswith("#")]
    got = [int(x) for x in rng.splitmix64_stream(1234567, len(want))]
    assert got == want


def test_rademacher_entries_and_balance():
    X = rng.rademacher(7, 20000, 0, 8)
    assert set(np.unique(X)) == {-1.0, 1.0}
    # each column is balanced to within 5 standard deviations
    assert np.all(np.abs(X.sum(axis=0)) < 5 * np.sqrt(20000))
    # distinct columns are nearly orthogonal (E[x x^T] = I)
    G = X.T @ X / 20000
    assert np.allclose(np.diag(G), 1.0)
    assert np.max(np.abs(G - np.eye(8))) < 5 / np.sqrt(20000)


def test_rademacher_columns_are_addressed_globally():
    A = rng.rademacher(3, 100, 0, 10)
    B = rng.rademacher(3, 100, 4, 3)
    assert np.array_equal(A[:, 4:7], B)
    C = rng.rademacher(4, 100, 0, 10)
    assert not np.array_equal(A, C)


def test_rademacher_row_relabelling():
    perm = np.random.default_rng(0).permutation(50)
    A = rng.rademacher(9, 50, 0, 4)
    B = rng.rademacher(9, 50, 0, 4, rows=perm)
    assert np.array_equal(A[perm], B)
