"""Pins for oracle.strang: closed forms, invariants, special cases (no GPU)."""

import math

import numpy as np
import pytest

from oracle import lattice as L
from oracle import strang as S
import workloads as w

CASES = [
    (np.array([1, 34]), (55,)),                       # Sec. 2.1 worked example
    (np.array([1, 7, 11]), (64,)),
    (np.array([[1, 0], [3, 1]]), (12, 6)),            # rank-2, canonical
    (np.array([[1, 0, 0], [1, 1, 6], [6, 4, 0], [0, 2, 3]]), (8, 4, 2)),   # rank-3 (Sec. 2.5), canonical
]


def _setup(Z, n):
    dp, _ = L.minl2_norms_dp(Z, n)
    H, _ = L.minl2_by_enumeration(Z, n, math.sqrt(dp.max()) + 1e-9)
    P = L.lattice_points(Z, n)
    return dp, H, P


def _rand_c(rng, m):
    return rng.standard_normal(m) + 1j * rng.standard_normal(m)


@pytest.mark.parametrize("Z,n", CASES)
def test_fft_coeffs_equal_direct_lattice_rule(Z, n):
    """Thm 1(iii): the r-D FFT in bin order equals the lattice rule of eq. approx_uhat,
    evaluated directly with the vectors h_chi (no residue map)."""
    dp, H, P = _setup(Z, n)
    rng = np.random.default_rng(0)
    u = _rand_c(rng, P.shape[0])
    direct = S.lattice_rule_coeffs(u, P, H)
    assert np.allclose(S.coeffs(u, n), direct, atol=1e-12)


@pytest.mark.parametrize("Z,n", CASES)
def test_interpolation_property(Z, n):
    """Thm 1(ii): u_a(p) = u(p) at lattice points, u_a = sum_h uhat_a(h) exp(2 pi i h.x)."""
    dp, H, P = _setup(Z, n)
    u = _rand_c(np.random.default_rng(1), P.shape[0])
    uh = S.coeffs(u, n)
    ua = np.exp(2j * np.pi * (P @ H.T)) @ uh
    assert np.allclose(ua, u, atol=1e-11)
    assert np.allclose(S.samples(uh, n), u, atol=1e-12)


def _trig_state(H, P, rng, k=8):
    """u0 = sum of k plane waves from the anti-aliasing set, and its data."""
    idx = rng.choice(H.shape[0], size=k, replace=False)
    c = _rand_c(rng, k)
    hs = H[idx]
    return hs, c


@pytest.mark.parametrize("Z,n", CASES)
@pytest.mark.parametrize("gamma", [0.1, 1.0])
def test_free_evolution_exact(Z, n, gamma):
    """v = 0: the TDSE solution for u0 = sum c_h e^{2 pi i h.x} is
    sum c_h exp(-i gamma 2 pi^2 |h|^2 t) e^{2 pi i h.x} (Lemma 1, eq. Fourier-ODE with f = 0)."""
    dp, H, P = _setup(Z, n)
    rng = np.random.default_rng(2)
    hs, c = _trig_state(H, P, rng)
    E = np.exp(2j * np.pi * (P @ hs.T))
    u0 = E @ c
    T, N = 0.37, 13
    exact = E @ (c * np.exp(-1j * gamma * 2 * np.pi ** 2 * (hs * hs).sum(1) * T))
    u = S.strang(u0, np.zeros(P.shape[0]), dp, n, gamma, T / N, N)
    assert np.allclose(u, exact, atol=1e-11)


@pytest.mark.parametrize("Z,n", CASES)
def test_constant_potential_global_phase(Z, n):
    """v = c: A and B commute (Sec. 2.3), the solution is free evolution times exp(-i c t / gamma)."""
    dp, H, P = _setup(Z, n)
    rng = np.random.default_rng(3)
    hs, cc = _trig_state(H, P, rng)
    E = np.exp(2j * np.pi * (P @ hs.T))
    u0 = E @ cc
    gamma, T, N, cst = 0.3, 0.5, 7, 2.75
    exact = E @ (cc * np.exp(-1j * gamma * 2 * np.pi ** 2 * (hs * hs).sum(1) * T)) * np.exp(
        -1j * cst * T / gamma)
    u = S.strang(u0, np.full(P.shape[0], cst), dp, n, gamma, T / N, N)
    assert np.allclose(u, exact, atol=1e-11)


def test_norm_conserved_and_time_reversible():
    """Thm 3 / Sec. 3.3: every factor is unitary, so ||u|| is conserved; S(-dt) S(dt) = I."""
    inst = w.c2(12)
    n = inst.n
    P = L.lattice_points(inst.Z, n)
    dp, _ = L.minl2_norms_dp(inst.Z, n)
    v, u0 = inst.v(P), inst.u0(P)
    u = S.strang(u0, v, dp, n, inst.gamma, 1e-2, 200)
    assert abs(S.norm2(u) - S.norm2(u0)) < 1e-12
    back = S.strang(u, v, dp, n, inst.gamma, -1e-2, 200)
    assert np.allclose(back, u0, atol=1e-11)


def test_second_order_convergence():
    """Thm 3(ii), Sec. 3.2: global error O(dt^2) against a fine-step reference (T = 1)."""
    z, n = np.array([1, 21]), (89,)
    P = L.lattice_points(z, n)
    dp, _ = L.minl2_norms_dp(z, n)
    gamma = 0.5
    v = w.v_smooth(P)
    u0 = w.gaussian_packet(P, 0.15, [0.5, 0.5])
    ref = S.strang(u0, v, dp, n, gamma, 1.0 / 10000, 10000)
    errs = []
    for m in (20, 40, 80, 160):
        u = S.strang(u0, v, dp, n, gamma, 1.0 / m, m)
        errs.append(np.sqrt(np.mean(np.abs(u - ref) ** 2)))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    for r in ratios:
        assert 3.6 < r < 4.4, ratios


def _dense_ops(Z, n, v_fun, gamma):
    """Unitary lattice Fourier matrix F (rows h_chi, cols p_kappa) built from its definition,
    D_n and W_n = F V_n F^H (eq. ode, eq. Dn, eq. Vn, Lemma 3)."""
    dp, H, P = _setup(Z, n)
    N = P.shape[0]
    F = np.exp(-2j * np.pi * (H @ P.T)) / math.sqrt(N)
    V = np.diag(v_fun(P))
    W = F @ V @ F.conj().T
    D = np.diag(4 * np.pi ** 2 * (H * H).sum(1).astype(float))
    return F, D, W, H, P, dp


def test_strang_converges_to_dense_semidiscrete_propagator():
    """The Strang step approximates exp(-i (W/gamma + gamma D/2) t) (eq. ode and its exact
    solution, Sec. 2.4) with O(dt^2) error; dense eigen-decomposition at n = 55."""
    Z, n = np.array([1, 34]), (55,)
    gamma, T = 0.5, 1.0
    F, D, W, H, P, dp = _dense_ops(Z, n, w.v_smooth, gamma)
    A = W / gamma + gamma * D / 2
    lam, Q = np.linalg.eigh(A)
    u0 = w.gaussian_packet(P, 0.2, [0.5, 0.5], k0=1)
    uh0 = F @ u0 / math.sqrt(P.shape[0])            # coefficients, eq. approx_uhat
    exact_h = Q @ (np.exp(-1j * lam * T) * (Q.conj().T @ uh0))
    errs = []
    for m in (20, 40, 80, 160):
        u = S.strang(u0, w.v_smooth(P), dp, n, gamma, T / m, m)
        uh = F @ u / math.sqrt(P.shape[0])
        errs.append(np.linalg.norm(uh - exact_h))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert errs[-1] < 1e-3
    for r in ratios:
        assert 3.5 < r < 4.5, ratios


def test_multiplication_operator_is_circulant():
    """Lemma 3: W_n = F V_n F^H is circulant with w_{xi-xi'} = sum over h.z = xi-xi' of vhat(h),
    here for v = 1 + 0.4 cos 2 pi x_1 + 0.25 cos 2 pi (x_1 + 2 x_2)."""
    Z, n = np.array([1, 34]), (55,)

    def v_fun(P):
        return 1 + 0.4 * np.cos(2 * np.pi * P[:, 0]) + 0.25 * np.cos(2 * np.pi * (P[:, 0] + 2 * P[:, 1]))

    F, D, W, H, P, dp = _dense_ops(Z, n, v_fun, 1.0)
    chi = L.chi_index(H, Z, n)
    order = np.argsort(chi)
    Wb = W[np.ix_(order, order)]                         # rows/cols by bin xi
    N = 55
    vhat = {(0, 0): 1.0, (1, 0): 0.2, (-1, 0): 0.2, (1, 2): 0.125, (-1, -2): 0.125}
    wv = np.zeros(N, dtype=complex)
    for h, c in vhat.items():
        wv[(h[0] * 1 + h[1] * 34) % N] += c
    expected = np.array([[wv[(a - b) % N] for b in range(N)] for a in range(N)])
    assert np.allclose(Wb, expected, atol=1e-12)


def test_regular_grid_equals_textbook_split_step():
    """Rank-2 lattice with Z = I, n = (N, N) is the regular grid (Sec. 2.1); the step is the
    classic split-step Fourier method, written here with fftfreq wave numbers."""
    N = 16
    Z, n = np.eye(2, dtype=np.int64), (N, N)
    P = L.lattice_points(Z, n)
    dp, _ = L.minl2_norms_dp(Z, n)
    gamma, dt, steps = 0.2, 0.01, 25
    v = w.v_harmonic(P)
    u0 = w.gaussian_packet(P, 0.12, [0.45, 0.55], k0=2)
    out = S.strang(u0, v, dp, n, gamma, dt, steps)
    kx = np.fft.fftfreq(N, d=1.0 / N)
    k2 = kx[:, None] ** 2 + kx[None, :] ** 2
    kin = np.exp(-1j * gamma * 2 * np.pi ** 2 * k2 * dt)
    half = np.exp(-1j * dt * v.reshape(N, N) / (2 * gamma))
    u = u0.reshape(N, N)
    for _ in range(steps):
        u = half * u
        u = np.fft.ifft2(kin * np.fft.fft2(u))
        u = half * u
    # fftfreq puts the Nyquist wave number at -N/2; |h|^2 is the same for +-N/2
    assert np.allclose(out, u.reshape(-1), atol=1e-12)


def test_regular_3d_grid_equals_textbook_split_step():
    """Rank-3 lattice with Z = I, n = (N, N, N/2) is a regular 3-D grid (Sec. 2.1, 2.5): the step is
    the classic split-step Fourier method over a 3-D array, with fftfreq wave numbers."""
    n = (8, 8, 4)
    Z = np.eye(3, dtype=np.int64)
    P = L.lattice_points(Z, n)
    dp, _ = L.minl2_norms_dp(Z, n)
    gamma, dt, steps = 0.15, 0.01, 20
    v = w.v_harmonic(P)
    u0 = w.gaussian_packet(P, 0.15, [0.45, 0.55, 0.5], k0=1)
    out = S.strang(u0, v, dp, n, gamma, dt, steps)
    k = [np.fft.fftfreq(m, d=1.0 / m) for m in n]
    k2 = k[0][:, None, None] ** 2 + k[1][None, :, None] ** 2 + k[2][None, None, :] ** 2
    kin = np.exp(-1j * gamma * 2 * np.pi ** 2 * k2 * dt)
    half = np.exp(-1j * dt * v.reshape(n) / (2 * gamma))
    u = u0.reshape(n)
    for _ in range(steps):
        u = half * u
        u = np.fft.ifftn(kin * np.fft.fftn(u))
        u = half * u
    # the Nyquist wave number -N/2 of fftfreq has the same |h|^2 as +N/2
    assert np.allclose(out, u.reshape(-1), atol=1e-12)


def test_energy_nearly_conserved():
    """Sec. 3.3: <Hu, u> is conserved by the exact flow; Strang keeps it to O(dt^2)."""
    inst = w.c2(12)
    n = inst.n
    P = L.lattice_points(inst.Z, n)
    dp, _ = L.minl2_norms_dp(inst.Z, n)
    v, u0 = inst.v(P), inst.u0(P)
    E0 = S.energy(u0, v, dp, n, inst.gamma)
    u = S.strang(u0, v, dp, n, inst.gamma, 1e-3, 300)
    E1 = S.energy(u, v, dp, n, inst.gamma)
    assert abs(E1 - E0) / abs(E0) < 1e-4


def test_adjoint_gradient_matches_finite_differences():
    """Adjoint gradient of J = |<u_N, phi>|^2 against central differences (FP64)."""
    z, n = np.array([1, 7, 11]), (64,)
    P = L.lattice_points(z, n)
    dp, _ = L.minl2_norms_dp(z, n)
    gamma, dt, N = 0.2, 0.02, 9
    v = w.v_smooth(P)
    u0 = w.gaussian_packet(P, 0.2, [0.5, 0.5, 0.5], k0=1)
    phi = w.gaussian_packet(P, 0.2, [0.6, 0.5, 0.5])
    J, gv, gu, uN = S.strang_adjoint(u0, v, dp, n, gamma, dt, N, phi, ckpt=4)
    assert np.isclose(J, S.overlap_objective(S.strang(u0, v, dp, n, gamma, dt, N), phi))
    rng = np.random.default_rng(5)
    f = lambda vv, uu: S.overlap_objective(S.strang(uu, vv, dp, n, gamma, dt, N), phi)
    eps = 1e-6
    for _ in range(3):
        dv = rng.standard_normal(v.size)
        fd = (f(v + eps * dv, u0) - f(v - eps * dv, u0)) / (2 * eps)
        assert abs(fd - gv @ dv) < 1e-7 * max(1.0, abs(fd))
        du = _rand_c(rng, u0.size)
        fd = (f(v, u0 + eps * du) - f(v, u0 - eps * du)) / (2 * eps)
        an = np.real(np.conj(gu) @ du)        # dJ = Re(conj(g) . du)
        assert abs(fd - an) < 1e-7 * max(1.0, abs(fd))


def test_adjoint_checkpoint_stride_invariance():
    z, n = np.array([1, 7, 11]), (64,)
    P = L.lattice_points(z, n)
    dp, _ = L.minl2_norms_dp(z, n)
    v = w.v_smooth(P)
    u0 = w.gaussian_packet(P, 0.2, [0.5, 0.5, 0.5])
    phi = w.gaussian_packet(P, 0.2, [0.6, 0.5, 0.5])
    a = S.strang_adjoint(u0, v, dp, n, 0.1, 0.01, 10, phi, ckpt=1)
    b = S.strang_adjoint(u0, v, dp, n, 0.1, 0.01, 10, phi, ckpt=7)
    assert np.allclose(a[1], b[1], atol=1e-14) and np.allclose(a[2], b[2], atol=1e-14)


# --------------------------------------------------------------------------
# Spot-check helpers (coeff_at, plane_wave_evolution)
# --------------------------------------------------------------------------
RANK2_SMALL = [(w.c5(10, 8, 16, 6).Z, (1024, 256))]


@pytest.mark.parametrize("Z,n", CASES + RANK2_SMALL)
def test_coeff_at_equals_direct_lattice_rule(Z, n):
    """coeff_at (multi-index form, integer-reduced exponents) equals eq. approx_uhat summed
    over the lattice points with the vectors h themselves."""
    P = L.lattice_points(Z, n)
    rng = np.random.default_rng(5)
    u = _rand_c(rng, P.shape[0])
    d = P.shape[1]
    H = rng.integers(-3, 4, size=(6, d))
    xi = L.residues(H, Z, n)
    got = S.coeff_at(u, n, xi)
    assert np.allclose(got, S.lattice_rule_coeffs(u, P, H), rtol=0, atol=1e-12 * np.abs(u).max())


@pytest.mark.parametrize("Z,n", CASES + RANK2_SMALL)
def test_plane_wave_evolution_equals_strang_run(Z, n):
    """Closed-form constant-potential evolution of a few plane waves equals the FFT Strang loop."""
    norms, _ = L.minl2_norms_dp(Z, n)
    rng = np.random.default_rng(6)
    N = int(np.prod(n))
    bins = rng.choice(N, size=5, replace=False)
    xi = np.stack(np.unravel_index(bins, n), axis=1)
    c = _rand_c(rng, 5)
    u0 = w.plane_waves(xi, c, n)
    gamma, dt, nsteps, vc = 0.1, 2e-3, 40, 0.7
    ref = S.strang(u0, np.full(N, vc), norms, n, gamma, dt, nsteps)
    kappa = np.stack(np.unravel_index(np.arange(N), n), axis=1)
    got = S.plane_wave_evolution(xi, norms[bins], c, n, gamma, dt, nsteps, vc, kappa)
    assert np.allclose(got, ref, rtol=0, atol=1e-11)


def test_c5_small_norm_vectors_are_their_bins_representatives():
    """For the C5 lattice (HC bound 16, d = 16) every h with ||h||^2 <= 4 lies in the hyperbolic
    cross, on which h -> xi is injective, so h is the unique minimal-norm vector of its bin:
    the min-l2 norm of its bin is ||h||^2.  Checked here on the full-size generating vectors."""
    inst = w.c5()
    B = L.ball_points(16, 2.0)
    HC = w.hyperbolic_cross(16, 16)
    hc = {tuple(r) for r in HC.tolist()}
    assert all(tuple(r) in hc for r in B.tolist())
    xi = L.residues(HC, inst.Z, inst.n)
    keys = xi[:, 0] * inst.n[1] + xi[:, 1]
    assert np.unique(keys).size == HC.shape[0]


def test_composed_strang_single_weight_is_strang():
    Z, n = np.array([1, 7, 11]), (64,)
    dp, H, P = _setup(Z, n)
    u0 = w.gaussian_packet(P, 0.2, [0.5] * 3)
    v = w.v_smooth(P)
    a = S.strang_composed(u0, v, dp, n, 0.3, 0.01, 7, [1.0])
    b = S.strang(u0, v, dp, n, 0.3, 0.01, 7)
    assert np.allclose(a, b, rtol=0, atol=1e-14)


def test_composed_strang_fourth_order_against_dense_propagator():
    """The triple (c, 1 - 2c, c), c = 1/(2 - 2^(1/3)), converges with O(dt^4) to the exact
    semi-discrete propagator exp(-i (W/gamma + gamma D/2) t) (dense eigen-decomposition, n = 55)."""
    Z, n = np.array([1, 34]), (55,)
    gamma, T = 0.5, 1.0
    F, D, W, H, P, dp = _dense_ops(Z, n, w.v_smooth, gamma)
    lam, Q = np.linalg.eigh(W / gamma + gamma * D / 2)
    u0 = w.gaussian_packet(P, 0.2, [0.5, 0.5], k0=1)
    exact = F.conj().T @ (Q @ (np.exp(-1j * lam * T) * (Q.conj().T @ (F @ u0))))      # F is unitary
    c = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
    errs = []
    for m in (80, 160, 320):                       # dt |lambda|_max <= 2.3: the asymptotic range
        u = S.strang_composed(u0, w.v_smooth(P), dp, n, gamma, T / m, m, [c, 1 - 2 * c, c])
        errs.append(np.linalg.norm(u - exact) / np.linalg.norm(exact))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert errs[-1] < 1e-6
    for r in ratios:
        assert 13 < r < 19, (errs, ratios)


@pytest.mark.parametrize("Z,n", CASES)
@pytest.mark.parametrize("gamma,c0", [(0.5, 0.0), (0.1, 1.7), (2.0, -0.6)])
def test_energy_of_plane_waves_closed_form(Z, n, gamma, c0):
    """Sec. 3.3 energy <H u, u>, H = -(gamma/2) Lap + v / gamma, on a trigonometric state.

    For u = sum_j c_j exp(2 pi i h_j . x) with distinct anti-aliasing vectors h_j and a
    constant potential v = c0, the Laplacian acts on each plane wave by -4 pi^2 ||h_j||^2
    and the waves are orthonormal under the lattice rule, so
        E = sum_j |c_j|^2 (2 pi^2 gamma ||h_j||^2 + c0 / gamma)
    exactly.  This fixes the absolute scale of both terms (a common factor would
    pass every conservation test)."""
    dp, H, P = _setup(Z, n)
    rng = np.random.default_rng(11)
    for k in (1, 3):
        idx = rng.choice(H.shape[0], size=k, replace=False)
        hs = H[idx]
        c = _rand_c(rng, k)
        u = np.exp(2j * np.pi * (P @ hs.T)) @ c
        v = np.full(P.shape[0], c0)
        h2 = np.sum(hs.astype(np.float64) ** 2, axis=1)
        expect = float(np.sum(np.abs(c) ** 2 * (2.0 * np.pi ** 2 * gamma * h2 + c0 / gamma)))
        got = S.energy(u, v, dp, n, gamma)
        assert abs(got - expect) <= 1e-11 * max(1.0, abs(expect)), (got, expect)
    # a single zero-frequency wave isolates the potential term, a single wave with v = 0
    # the kinetic term
    u0 = np.full(P.shape[0], 2.0 + 0j)
    assert abs(S.energy(u0, np.full(P.shape[0], c0), dp, n, gamma) - 4.0 * c0 / gamma) < 1e-12
    j = int(np.argmax(np.sum(H.astype(np.float64) ** 2, axis=1)))
    u1 = np.exp(2j * np.pi * (P @ H[j]))
    want = 2.0 * np.pi ** 2 * gamma * float(np.sum(H[j].astype(np.float64) ** 2))
    assert abs(S.energy(u1, np.zeros(P.shape[0]), dp, n, gamma) - want) < 1e-10 * want
