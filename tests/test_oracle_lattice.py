"""Pins for oracle.lattice against the paper's theorems and brute force (no GPU)."""

import itertools
import math

import numpy as np
import pytest

from oracle import lattice as L
import workloads as w

pytestmark = pytest.mark.filterwarnings("ignore")

# (Z, n) test lattices: the paper's worked example n=55, z=(1,34) (Sec. 2.1, Fig. 1),
# small rank-1 lattices, rank-2 and rank-3 lattices in canonical form and regular grids.
RANK1 = [
    (np.array([1, 34]), (55,)),
    (np.array([1, 5]), (32,)),
    (np.array([1, 7, 11]), (64,)),
    (np.array([1, 5, 7, 11]), (81,)),
    (np.array([1, 31]), (961,)),
]
RANK2 = [
    (np.array([[1, 0], [3, 1]]), (12, 6)),
    (np.array([[1, 0], [5, 1], [7, 3]]), (16, 4)),
    (np.eye(2, dtype=np.int64), (8, 8)),            # regular grid (r = d, Z = I)
]
# rank 3 (Sec. 2.5): seeded lattices whose N points are distinct (Def. 1), and a 3-D grid
RANK3 = [
    (np.array([[1, 0, 0], [1, 1, 6], [6, 4, 0], [0, 2, 3]]), (8, 4, 2)),
    (np.array([[1, 0, 0], [0, 4, 4], [0, 0, 2], [2, 5, 3]]), (6, 6, 3)),
    (np.eye(3, dtype=np.int64), (4, 4, 2)),
]


def _box(d, half):
    return np.array(list(itertools.product(range(-half, half + 1), repeat=d)), dtype=np.int64)


@pytest.mark.parametrize("Z,n", RANK1 + RANK2 + RANK3)
def test_character_property(Z, n):
    """eq. char: (1/N) sum_p exp(2 pi i h.p) = 1 if h in the dual lattice, else 0."""
    P = L.lattice_points(Z, n)
    d = P.shape[1]
    H = _box(d, 3 if d <= 3 else 2)
    s = np.exp(2j * np.pi * (H @ P.T)).mean(axis=1)
    dual = L.in_dual(H, Z, n)
    # membership by the definition Z^T h = 0 (mod n), written out independently
    Zm = np.asarray(Z).reshape(d, -1)
    nn = np.array(n)
    dual_def = np.all(((H @ Zm) % nn) == 0, axis=1)
    assert np.array_equal(dual, dual_def)
    assert np.allclose(s[dual], 1.0, atol=1e-12)
    assert np.allclose(s[~dual], 0.0, atol=1e-12)


@pytest.mark.parametrize("Z,n", RANK1 + RANK2 + RANK3)
def test_points_distinct_and_canonical(Z, n):
    """Def. 1: a canonical lattice has prod n_i distinct points in [0,1)^d."""
    P = L.lattice_points(Z, n)
    N = int(np.prod(n))
    assert P.shape[0] == N
    assert np.all((P >= 0) & (P < 1))
    assert np.unique(np.round(P * N).astype(np.int64), axis=0).shape[0] == N
    assert L.is_canonical(Z, n)


def test_rank1_points_closed_form():
    """Sec. 2.1: p_k = frac(k z / n) for a rank-1 lattice, k = 0..n-1."""
    z, n = np.array([1, 34]), 55
    P = L.lattice_points(z, (n,))
    for k in (0, 1, 2, 17, 54):
        assert np.allclose(P[k], [(k * 1 % n) / n, (k * 34 % n) / n])


def test_not_canonical_detected():
    assert not L.is_canonical(np.array([2, 4]), (8,))          # only 4 distinct points
    assert not L.is_canonical(np.array([[1, 1], [1, 1]]), (6, 4))  # 4 does not divide 6


def _bruteforce_min_norms(Z, n, half):
    """min ||h||^2 per bin over the box |h_j| <= half, by exhaustive search."""
    Zm = np.asarray(Z).reshape(-1, len(n))
    d = Zm.shape[0]
    N = int(np.prod(n))
    best = np.full(N, np.iinfo(np.int64).max)
    H = _box(d, half)
    xi = (H @ Zm) % np.array(n)
    chi = np.zeros(H.shape[0], dtype=np.int64)
    for i, ni in enumerate(n):
        chi = chi * ni + xi[:, i]
    nr = (H * H).sum(axis=1)
    np.minimum.at(best, chi, nr)
    return best


@pytest.mark.parametrize("Z,n", RANK1 + RANK2 + RANK3)
def test_minl2_dp_equals_paper_recipe_and_bruteforce(Z, n):
    """eq. hrepresenter: DP norms = the paper's sort-and-greedy recipe (Sec. 3.1) = exhaustive minimum."""
    N = int(np.prod(n))
    d = np.asarray(Z).reshape(-1, len(n)).shape[0]
    dp, box = L.minl2_norms_dp(Z, n)
    radius = math.sqrt(dp.max()) + 1e-9
    H, en = L.minl2_by_enumeration(Z, n, radius)
    assert np.array_equal(dp, en)
    half = int(math.ceil(math.sqrt(dp.max())))
    bf = _bruteforce_min_norms(Z, n, half)
    assert np.array_equal(dp, bf)
    # the recipe's set is a full anti-aliasing set (Def. 2) with h_chi in bin chi
    assert H.shape == (N, d)
    assert L.is_anti_aliasing(H, Z, n)
    assert np.array_equal(L.chi_index(H, Z, n), np.arange(N))


def test_minl2_dp_c2_sample_against_bruteforce_per_bin():
    """At the n = 2^22, d = 6 size: sampled bins against an exhaustive per-bin search."""
    inst = w.c2(22)
    n = inst.n
    z = inst.Zmat[:, 0]
    dp, box = L.minl2_norms_dp(inst.Z, n)
    assert dp.max() <= (box + 1) ** 2
    R = int(math.ceil(math.sqrt(dp.max())))
    B = L.ball_points(6, R)
    res = (B @ z) % n[0]
    nr = (B * B).sum(axis=1)
    best = np.full(n[0], np.iinfo(np.int64).max)
    np.minimum.at(best, res, nr)
    assert np.array_equal(best, dp)


def test_c1_box_is_full_anti_aliasing_and_minl2():
    """C1: the box |h_j| <= 15 is a full anti-aliasing set for z=(1,31), n=961, and it
    is minimal in l2 bin by bin (so EXPLICIT and MINL2 agree on ||h_chi||^2)."""
    inst = w.c1()
    I = inst.index_set
    assert I.shape == (961, 2)
    assert L.is_anti_aliasing(I, inst.Z, inst.n)
    ex = L.explicit_norms(I, inst.Z, inst.n)
    dp, _ = L.minl2_norms_dp(inst.Z, inst.n)
    assert np.array_equal(ex, dp)


def test_explicit_rejects_aliasing_set():
    z, n = np.array([1, 34]), (55,)
    I = np.array([[0, 0], [55, 0]] + [[k, 0] for k in range(1, 54)])
    with pytest.raises(ValueError):
        L.explicit_norms(I, z, n)


def test_regular_grid_minl2_is_symmetric_box():
    """Regular grid (r = d, Z = I, Sec. 2.1): the minimal set is the centred box per axis."""
    N = 8
    dp, _ = L.minl2_norms_dp(np.eye(3, dtype=np.int64), (N, N, N))
    a = np.arange(N)
    m1 = np.minimum(a, N - a) ** 2
    exp = (m1[:, None, None] + m1[None, :, None] + m1[None, None, :]).reshape(-1)
    assert np.array_equal(dp, exp)


@pytest.mark.parametrize("Z,n", [RANK1[0], RANK1[2], RANK2[0], RANK3[0], RANK3[1]])
def test_dual_character_property(Z, n):
    """Thm 1(i): (1/N) sum_{h in A} exp(2 pi i h.(p - p')) = delta_{p,p'} for a full A."""
    dp, _ = L.minl2_norms_dp(Z, n)
    H, _ = L.minl2_by_enumeration(Z, n, math.sqrt(dp.max()) + 1e-9)
    P = L.lattice_points(Z, n)
    M = np.exp(2j * np.pi * (H @ P.T))                 # (chi, kappa)
    G = (M.conj().T @ M) / P.shape[0]
    assert np.allclose(G, np.eye(P.shape[0]), atol=1e-10)


def test_table1_generating_vectors_are_units():
    """Table 1 lattices (golden fixture): every component is a unit mod n = 2^m."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_generating_vectors.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 5
    for row in rows:
        d, m = int(row[0]), int(row[1])
        z = np.array([int(x) for x in row[2:]], dtype=np.int64)
        assert z.size >= d and z[0] == 1
        assert np.all(z % 2 == 1)


# ---------------------------------------------------------------------------
# component-by-component reconstructing lattice (Sec. 3.1 search, Def. 2 test)
# ---------------------------------------------------------------------------
def _collides(proj, z, n):
    """Pure-Python pair search: two distinct projected rows with the same bin."""
    nt = [int(x) for x in np.atleast_1d(n)]
    rows = sorted({tuple(int(v) for v in p) for p in proj})
    seen = {}
    for p in rows:
        key = tuple(sum(p[i] * int(z[i][q]) for i in range(len(p))) % nt[q] for q in range(len(nt)))
        if key in seen:
            return True
        seen[key] = p
    return False


@pytest.mark.parametrize("n", [128, (16, 16), 192])
def test_cbc_accepts_first_injective_candidate_brute_force(n):
    import workloads as w
    rng = np.random.default_rng(5)
    I = rng.integers(-3, 4, size=(30, 3))
    I = np.concatenate([I, I[:5]])                       # repeated rows are allowed
    r = len(np.atleast_1d(n))
    cand = w.cbc_candidates(3, n, 60, w.Rng(2, 11))
    Z, fixed = L.cbc_reconstructing(I, n, cand)
    assert fixed == 3
    assert Z[0, 0] == 1 and (r == 1 or Z[0, 1] == 0)
    rejected = 0
    for j in (1, 2):
        proj = I[:, : j + 1]
        t = next(t for t in range(cand.shape[1]) if np.array_equal(cand[j - 1, t], Z[j]))
        rejected += t
        for tt in range(t):                               # every earlier candidate collides
            zz = np.concatenate([Z[:j], cand[j - 1, tt][None]])
            assert _collides(proj, zz, n)
        assert not _collides(proj, Z[: j + 1], n)
    assert rejected >= 15                                 # the search passed over colliding candidates
    assert L.is_anti_aliasing(np.unique(I, axis=0), Z[:, 0] if r == 1 else Z, n)


def test_cbc_regular_grid_closed_form():
    """The box {0..a-1}^d is mapped injectively by z = (1, a, a^2, ...) mod a^d (mixed radix);
    z_j = 1 merges (1, 0, ..) and (0, 1, ..), so the search passes over it."""
    a, d = 4, 3
    I = np.array(np.meshgrid(*[np.arange(a)] * d, indexing="ij")).reshape(d, -1).T
    cand = np.array([[[1], [a]], [[a], [a * a]]])
    Z, fixed = L.cbc_reconstructing(I, a ** d, cand)
    assert fixed == d and list(Z[:, 0]) == [1, a, a * a]


def test_cbc_reports_a_component_without_injective_candidate():
    I = np.array([[0, 0], [1, 0], [0, 1]])
    Z, fixed = L.cbc_reconstructing(I, 8, np.array([[[1], [9]]]))    # 9 = 1 mod 8: (1,0), (0,1) share a bin
    assert fixed == 1 and list(Z[:, 0]) == [1, 0]
