"""Component-by-component reconstructing lattices on the GPU (lsp_cbc_reconstructing) against the
oracle's search on the same candidate lists (GB300)."""

import numpy as np
import pytest

from oracle import lattice as L
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [128, (16, 16), 192, 4096])
def test_cbc_small_cases_equal_oracle(lib, n):
    rng = np.random.default_rng(5)
    I = rng.integers(-3, 4, size=(30, 3))
    I = np.concatenate([I, I[:5]])
    cand = w.cbc_candidates(3, n, 60, w.Rng(2, 11))
    Zg, fg = lib.cbc_reconstructing(I, n, cand)
    Zo, fo = L.cbc_reconstructing(I, n, cand)
    assert fg == fo == 3 and np.array_equal(Zg, Zo)


def test_cbc_regular_grid_and_failure(lib):
    a, d = 4, 3
    I = np.array(np.meshgrid(*[np.arange(a)] * d, indexing="ij")).reshape(d, -1).T
    Z, fixed = lib.cbc_reconstructing(I, a ** d, np.array([[[1], [a]], [[a], [a * a]]]))
    assert fixed == d and list(Z[:, 0]) == [1, a, a * a]
    Z, fixed = lib.cbc_reconstructing(np.array([[0, 0], [1, 0], [0, 1]]), 8, np.array([[[1], [9]]]))
    assert fixed == 1 and list(Z[:, 0]) == [1, 0]


def test_cbc_c2_index_set_full_size(lib):
    """C2's design set, the hyperbolic cross prod(1 + |h_j|) <= 64 in d = 6 (51,233 vectors), at
    n = 2^22: the GPU search and the oracle's agree, and the result maps the set injectively."""
    I = w.hyperbolic_cross(6, 64)
    n = 1 << 22
    cand = w.cbc_candidates(6, n, 400, w.Rng(0, 21))
    Zg, fg = lib.cbc_reconstructing(I, n, cand)
    Zo, fo = L.cbc_reconstructing(I, n, cand)
    assert fg == fo == 6 and np.array_equal(Zg, Zo)
    assert L.is_anti_aliasing(I, Zg[:, 0], (n,))


def test_cbc_rank2_equal_oracle(lib):
    """Rank 2, d = 16, the hyperbolic cross with bound 6 on 2^10 x 2^8 (the C5 family at reduced size)."""
    I = w.hyperbolic_cross(16, 6)
    n = (1 << 10, 1 << 8)
    cand = w.cbc_candidates(16, n, 64, w.Rng(1, 21))
    Zg, fg = lib.cbc_reconstructing(I, n, cand)
    Zo, fo = L.cbc_reconstructing(I, n, cand)
    assert fg == fo and np.array_equal(Zg, Zo)
    if fo == 16:
        assert L.is_anti_aliasing(I, Zg, n) and L.is_canonical(Zg, n)
