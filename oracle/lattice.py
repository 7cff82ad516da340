"""Lattices, bin maps and anti-aliasing sets (paper Sec. 2.1, Def. 1-2, Thm 1, Lemma 4).

Notation follows the paper: a rank-r lattice is given by generating vectors
Z = (z_1, ..., z_r) in Z^{d x r} (columns) and moduli n = (n_1, ..., n_r) with
n_{i+1} | n_i (canonical form, Def. 1).  A rank-1 lattice is the case r = 1.

Point order: kappa = sum_i kappa_i prod_{j>i} n_j (lexicographic, Sec. 2.5).
Bin order:   chi   = sum_i xi_i    prod_{j>i} n_j with xi_i = h.z_i mod n_i
             (Thm 1(iii), Sec. 2.5).
"""

from __future__ import annotations

import math
from typing import Sequence, Tuple

import numpy as np


def _as_Zn(Z, n) -> Tuple[np.ndarray, Tuple[int, ...]]:
    nt = tuple(int(x) for x in (n if isinstance(n, (tuple, list, np.ndarray)) else (n,)))
    Zm = np.asarray(Z, dtype=np.int64).reshape(-1, len(nt))
    return Zm, nt


def lattice_numerators(Z, n) -> np.ndarray:
    """Integer numerators q with p_kappa = q / N, N = prod n_i (Def. 1).

    p_kappa = (z_1 kappa_1 / n_1 + ... + z_r kappa_r / n_r) mod 1.  Since
    N / n_i is an integer, N p_kappa = sum_i z_i kappa_i (N / n_i) mod N exactly.
    """
    Zm, nt = _as_Zn(Z, n)
    N = int(np.prod(nt))
    grids = np.meshgrid(*[np.arange(ni, dtype=np.int64) for ni in nt], indexing="ij")
    kap = np.stack([g.reshape(-1) for g in grids], axis=1)        # (N, r), kappa_r fastest
    q = np.zeros((N, Zm.shape[0]), dtype=np.int64)
    for i, ni in enumerate(nt):
        mult = (Zm[:, i] % ni) * (N // ni)                           # (d,)
        q = (q + (kap[:, i:i + 1] * mult[None, :]) % N) % N
    return q


def lattice_points(Z, n) -> np.ndarray:
    """Lattice points p_kappa in [0,1)^d, shape (N, d), kappa lexicographic (Def. 1, Sec. 2.5)."""
    _, nt = _as_Zn(Z, n)
    N = int(np.prod(nt))
    return lattice_numerators(Z, n).astype(np.float64) / float(N)


def residues(h: np.ndarray, Z, n) -> np.ndarray:
    """xi = (h.z_1 mod n_1, ..., h.z_r mod n_r) for rows h, shape (m, r) (Def. 2, Thm 1(iii))."""
    Zm, nt = _as_Zn(Z, n)
    H = np.asarray(h, dtype=np.int64).reshape(-1, Zm.shape[0])
    return np.stack([(H @ Zm[:, i]) % nt[i] for i in range(len(nt))], axis=1)


def chi_index(h: np.ndarray, Z, n) -> np.ndarray:
    """Lexicographic bin number chi of each row h (Sec. 2.5)."""
    _, nt = _as_Zn(Z, n)
    xi = residues(h, Z, n)
    chi = np.zeros(xi.shape[0], dtype=np.int64)
    for i, ni in enumerate(nt):
        chi = chi * ni + xi[:, i]
    return chi


def in_dual(h: np.ndarray, Z, n) -> np.ndarray:
    """Membership in the dual lattice: Z^T h == 0 (mod n) (eq. dual)."""
    return np.all(residues(h, Z, n) == 0, axis=1)


def is_anti_aliasing(index_set: np.ndarray, Z, n) -> bool:
    """Def. 2: no two distinct h, h' in the set have Z^T (h - h') == 0 (mod n)."""
    chi = chi_index(index_set, Z, n)
    return np.unique(chi).size == chi.size


def is_canonical(Z, n) -> bool:
    """Def. 1, as read here: n_{i+1} | n_i and the N = prod n_i points are distinct.

    Def. 1 also asks every component of z_i to be prime to n_i; the paper's own
    regular grid (r = d, Z = I, Sec. 2.1) has zero components, so that clause is
    read as sufficient, not necessary, and the point count is what is checked.
    """
    Zm, nt = _as_Zn(Z, n)
    for i in range(len(nt) - 1):
        if nt[i] % nt[i + 1] != 0:
            return False
    q = lattice_numerators(Z, n)
    return np.unique(q, axis=0).shape[0] == q.shape[0]


# --------------------------------------------------------------------------
# Minimal-l2 anti-aliasing set (Lemma 4, eq. hrepresenter)
# --------------------------------------------------------------------------
def ball_points(d: int, radius: float) -> np.ndarray:
    """All h in Z^d with ||h||_2 <= radius (Sec. 3.1, step 1)."""
    R = int(math.floor(radius))
    r2 = radius * radius
    pts = [np.zeros((1, 0), dtype=np.int64)]
    partial = [np.zeros(1, dtype=np.int64)]
    cur, cs = pts[0], partial[0]
    for _ in range(d):
        rows, ss = [], []
        for a in range(-R, R + 1):
            s = cs + a * a
            keep = s <= r2
            if np.any(keep):
                sub = cur[keep]
                rows.append(np.concatenate([sub, np.full((sub.shape[0], 1), a, np.int64)], axis=1))
                ss.append(s[keep])
        cur = np.concatenate(rows, axis=0)
        cs = np.concatenate(ss)
    return cur


def minl2_by_enumeration(Z, n, radius: float):
    """The paper's construction of a full-cardinality anti-aliasing set (Sec. 3.1):

    1. generate all h with ||h||_2 <= radius,
    2. sort them by l2 norm, ascending,
    3. walk the sorted list, keeping h whenever its residue Z^T h mod n has not
       been seen, until n residues are covered.

    Ties in the norm are broken lexicographically on h (negative entries
    first); the resulting norms per bin do not depend on that choice.
    Returns (H, norms2): H[chi] is the representative of bin chi.
    Raises ValueError when the ball is too small to cover every bin.
    """
    Zm, nt = _as_Zn(Z, n)
    d = Zm.shape[0]
    N = int(np.prod(nt))
    B = ball_points(d, radius)
    nrm = np.einsum("ij,ij->i", B, B)
    order = np.lexsort(tuple(B[:, j] for j in range(d - 1, -1, -1)) + (nrm,))
    B, nrm = B[order], nrm[order]
    chi = chi_index(B, Z, n)
    H = np.zeros((N, d), dtype=np.int64)
    seen = np.zeros(N, dtype=bool)
    count = 0
    for t in range(B.shape[0]):
        c = chi[t]
        if not seen[c]:
            seen[c] = True
            H[c] = B[t]
            count += 1
            if count == N:
                break
    if count != N:
        raise ValueError("enumeration radius too small to fill every bin")
    return H, np.einsum("ij,ij->i", H, H)


def minl2_norms_dp(Z, n, box: int = 0):
    """min{ ||h||^2 : Z^T h == xi (mod n) } for every bin xi (eq. hrepresenter), exactly.

    Min-plus dynamic programme over the residue group Z_{n_1} x ... x Z_{n_r}:
        f_0 = [0 at xi = 0, +inf elsewhere]
        f_j(xi) = min_{|t| <= B} f_{j-1}(xi - t z_j mod n) + t^2
    gives the minimum over the box |h_j| <= B.  Any h outside the box has
    ||h||^2 >= (B+1)^2, so when max_xi f_d(xi) <= (B+1)^2 the box minimum is the
    minimum over all of Z^d.  Independently, h -/+ n_1 e_j stays in the class of
    h, so every minimiser has |h_j| <= n_1 / 2 and B >= n_1 // 2 always suffices.
    B starts from the radius of a ball holding N integer points and doubles
    until one of the two certificates holds.
    Returns (norms2 int64 array indexed by chi, B).
    """
    Zm, nt = _as_Zn(Z, n)
    d = Zm.shape[0]
    N = int(np.prod(nt))
    if box <= 0:
        vol1 = math.pi ** (d / 2) / math.gamma(d / 2 + 1)
        box = max(1, int(math.ceil((N / vol1) ** (1.0 / d))))
    INF = np.iinfo(np.int64).max // 4
    while True:
        f = np.full(nt, INF, dtype=np.int64)
        f[(0,) * len(nt)] = 0
        for j in range(d):
            g = np.full(nt, INF, dtype=np.int64)
            for t in range(-box, box + 1):
                shift = tuple(int((t * Zm[j, i]) % nt[i]) for i in range(len(nt)))
                # g(xi) <- f(xi - t z_j) + t^2 : roll f forward by t z_j
                np.minimum(g, np.roll(f, shift, axis=tuple(range(len(nt)))) + t * t, out=g)
            f = g
        if f.max() <= (box + 1) ** 2 or (box >= nt[0] // 2 and f.max() < INF):
            return f.reshape(-1), box
        if box >= nt[0] // 2:
            raise ValueError("bins unreachable: lattice not in canonical form")
        box = min(2 * box, nt[0] // 2)


def explicit_norms(index_set: np.ndarray, Z, n) -> np.ndarray:
    """||h_chi||^2 per bin for a caller-given full anti-aliasing set (Def. 2, |A| = n)."""
    _, nt = _as_Zn(Z, n)
    N = int(np.prod(nt))
    I = np.asarray(index_set, dtype=np.int64)
    if I.shape[0] != N:
        raise ValueError("index set must have exactly n elements")
    chi = chi_index(I, Z, n)
    if np.unique(chi).size != N:
        raise ValueError("index set is not anti-aliasing (Def. 2)")
    out = np.zeros(N, dtype=np.int64)
    out[chi] = np.einsum("ij,ij->i", I, I)
    return out


def explicit_table(index_set: np.ndarray, Z, n) -> np.ndarray:
    """Representative h_chi per bin for a caller-given full anti-aliasing set."""
    _, nt = _as_Zn(Z, n)
    I = np.asarray(index_set, dtype=np.int64)
    chi = chi_index(I, Z, n)
    H = np.zeros_like(I)
    H[chi] = I
    return H


# --------------------------------------------------------------------------
# Component-by-component reconstructing lattice (Sec. 3.1's CBC search, with
# injectivity of h -> bin on the index set, Def. 2 / Thm 1(iii), as the test)
# --------------------------------------------------------------------------
def cbc_reconstructing(index_set: np.ndarray, n, candidates) -> Tuple[np.ndarray, int]:
    """Component 0 fixed to 1 (rank 1) or (1, 0) (rank 2); component j takes the first
    candidate c of its list for which the bins of the distinct projections
    (h_0, ..., h_j) of the index set are distinct.

    candidates: array (d - 1, T, r); returns (Z of shape (d, r), number of components
    fixed).  When some component has no injective candidate, Z holds zeros from it on.
    """
    I = np.asarray(index_set, dtype=np.int64)
    nt = tuple(int(x) for x in np.atleast_1d(n))
    r = len(nt)
    d = I.shape[1]
    cand = np.asarray(candidates, dtype=np.int64).reshape(d - 1, -1, r)
    Z = np.zeros((d, r), dtype=np.int64)
    Z[0, 0] = 1
    for j in range(1, d):
        proj = np.unique(I[:, : j + 1], axis=0)
        for c in cand[j - 1]:
            Zj = Z[: j + 1].copy()
            Zj[j] = c
            chi = np.zeros(proj.shape[0], dtype=np.int64)
            for i, ni in enumerate(nt):
                chi = chi * ni + (proj @ Zj[:, i]) % ni
            if np.unique(chi).size == chi.size:
                Z[j] = c
                break
        else:
            return Z, j
    return Z, d
