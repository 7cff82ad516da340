"""Input generators: lattices in canonical form, fast field evaluation (no GPU)."""

import numpy as np
import pytest

from oracle import lattice as L
import workloads as w


@pytest.mark.parametrize("shape,bound", [((10, 8), 6), ((11, 9), 8), ((8, 6), 4)])
def test_rank2_generator_gives_canonical_injective_lattices(shape, bound):
    inst = w.c5(*shape, 16, bound)
    assert L.is_canonical(inst.Z, inst.n)
    assert L.is_anti_aliasing(w.hyperbolic_cross(16, bound), inst.Z, inst.n)


def test_units_in_every_component_merge_points_for_even_moduli():
    """Def. 1 asks each component of z_i to be prime to n_i; with n_1, n_2 even and every
    component odd the image of h -> (h.z_1, h.z_2) mod 2 is the diagonal, so the points
    k and k + (n_1/2, n_2/2) coincide and the lattice has fewer than n_1 n_2 points."""
    Z = np.array([[1, 3], [5, 7], [9, 1]])
    n = (16, 8)
    assert not L.is_canonical(Z, n)
    q = L.lattice_numerators(Z, n)
    k = np.array([8, 4])
    assert np.array_equal(q[k[0] * n[1] + k[1]], q[0])


def test_c5_fields_equal_direct_evaluation():
    inst = w.c5(10, 8, 16, 6)
    P = L.lattice_points(inst.Z, inst.n)
    v, u = w.c5_fields(inst, rows_per_chunk=100)
    assert np.allclose(v, inst.v(P), rtol=0, atol=1e-12)
    assert np.allclose(u, inst.u0(P), rtol=1e-12, atol=0)


def test_plane_waves_equal_exponentials_at_points():
    inst = w.c5(8, 6, 16, 4)
    P = L.lattice_points(inst.Z, inst.n)
    H = np.zeros((3, 16), dtype=np.int64)
    H[0, 0] = 1
    H[1, 3], H[1, 7] = 1, -1
    H[2, 12] = 2
    c = np.array([1.0, 0.5j, -0.25 + 0.1j])
    xi = L.residues(H, inst.Z, inst.n)
    got = w.plane_waves(xi, c, inst.n)
    ref = np.exp(2j * np.pi * (P @ H.T.astype(np.float64))) @ c
    assert np.allclose(got, ref, rtol=0, atol=1e-12)


def test_table1_vectors_match_the_golden_fixture():
    """The workload module's Table 1 vectors are the cited fixture's, row by row."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_generating_vectors.txt")
    rows = [list(map(int, ln.split())) for ln in open(path) if ln.strip() and not ln.startswith("#")]
    for r in rows:
        d, m, z = r[0], r[1], r[2:]
        if d <= 3:
            assert list(w.table1_z(d, m)) == z
        else:
            assert list(w.TABLE1_Z12) == z
            for dd in range(4, 13):
                assert list(w.table1_z(dd, 25)) == z[:dd]


def test_paper_initial_conditions():
    """g1 peaks at the packet centre (x_1 = 3/4, x_j = 1/2) and is separable; g2's factors are
    hats of half-width sqrt(gamma)/4 in x; both have unit lattice-rule norm."""
    inst = w.paper_instance(2, 18, init="g1", gamma=0.5)
    P = L.lattice_points(inst.Z, inst.n)
    g = inst.u0(P)
    assert abs(np.mean(np.abs(g) ** 2) - 1) < 1e-12
    k = int(np.argmax(np.abs(g)))
    assert np.allclose(P[k], [0.75, 0.5], atol=5e-3)
    gamma = 0.01
    h = w.paper_g2(P, gamma)
    assert abs(np.mean(np.abs(h) ** 2) - 1) < 1e-12 and np.all(h.real >= 0)
    far = np.abs(P[:, 1] - 0.5) > np.sqrt(gamma) / 4 + 1e-12
    assert np.all(h[far] == 0)


def test_cbc_candidates_are_seeded_units():
    """Candidate lists for the component-by-component search: shape (d - 1, count, r), every entry a
    unit modulo its n_i, the same lists for the same seed and different ones for another."""
    import math
    a = w.cbc_candidates(4, (1 << 10, 1 << 6), 50, w.Rng(3, 21))
    b = w.cbc_candidates(4, (1 << 10, 1 << 6), 50, w.Rng(3, 21))
    c = w.cbc_candidates(4, (1 << 10, 1 << 6), 50, w.Rng(4, 21))
    assert a.shape == (3, 50, 2) and np.array_equal(a, b) and not np.array_equal(a, c)
    assert all(math.gcd(int(x), 1 << 10) == 1 for x in a[..., 0].ravel())
    assert all(math.gcd(int(x), 1 << 6) == 1 for x in a[..., 1].ravel())
    r1 = w.cbc_candidates(3, 768, 40, w.Rng(0, 21))
    assert r1.shape == (2, 40, 1) and all(math.gcd(int(x), 768) == 1 for x in r1.ravel())
