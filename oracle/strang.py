"""Strang splitting on lattices (paper Sec. 2.2-2.5, eq. StrangTDSE, Algorithm 1), in FP64.

State convention: u holds the physical samples u(p_kappa) at the lattice
points, kappa lexicographic.  Spectral coefficients are the lattice-rule
coefficients of eq. approx_uhat,
    uhat_chi = (1/N) sum_kappa u_kappa exp(-2 pi i h_chi . p_kappa),
which by Thm 1(iii) equal the r-dimensional DFT of u (minus sign, eq. Fnx)
divided by N, with bins ordered lexicographically by xi = Z^T h mod n.

One Strang step (eq. StrangTDSE written in physical space by conjugating with
the Fourier matrix; Algorithm 1 loop body):
    u <- P o u,  uhat <- F u,  uhat_chi <- K_chi uhat_chi,  u <- F^{-1} uhat,  u <- P o u
with P_kappa = exp(-i dt v(p_kappa) / (2 gamma)) and
     K_chi   = exp(-i gamma 2 pi^2 ||h_chi||^2 dt).
The potential exponent carries 1/gamma as in eq. StrangTDSE and Lemma 1's
operator B = -(i/gamma) v; the kinetic phase follows eq. Fourier-ODE.
"""

from __future__ import annotations

import numpy as np


def _shape(n):
    return tuple(int(x) for x in (n if isinstance(n, (tuple, list, np.ndarray)) else (n,)))


# --------------------------------------------------------------------------
# Transforms (eq. approx_uhat, eq. Fnx, Thm 1(iii))
# --------------------------------------------------------------------------
def coeffs(u: np.ndarray, n) -> np.ndarray:
    """uhat = (1/N) * r-D DFT of u (minus sign), flattened lexicographically."""
    s = _shape(n)
    N = int(np.prod(s))
    return np.fft.fftn(np.asarray(u, dtype=np.complex128).reshape(s)).reshape(-1) / N


def samples(uhat: np.ndarray, n) -> np.ndarray:
    """Inverse of coeffs: u_kappa = sum_chi uhat_chi exp(+2 pi i h_chi . p_kappa)."""
    s = _shape(n)
    N = int(np.prod(s))
    return np.fft.ifftn(np.asarray(uhat, dtype=np.complex128).reshape(s)).reshape(-1) * N


def lattice_rule_coeffs(u: np.ndarray, points: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Direct lattice rule (eq. approx_uhat): (1/N) sum_p u(p) exp(-2 pi i h . p) for each row h.

    O(N * |H|): for small lattices only.  No residue map is involved.
    """
    ph = np.exp(-2j * np.pi * (np.asarray(H, dtype=np.float64) @ np.asarray(points).T))
    return ph @ np.asarray(u, dtype=np.complex128) / points.shape[0]


# --------------------------------------------------------------------------
# Phase factors (Algorithm 1: V_n, D_n diagonals)
# --------------------------------------------------------------------------
def kinetic_phase(norms2: np.ndarray, gamma: float, dt: float) -> np.ndarray:
    """exp(-i gamma/2 * D_n dt), D_n = diag(4 pi^2 ||h_chi||^2) (eq. Dn)."""
    return np.exp(-1j * (gamma / 2.0) * (4.0 * np.pi ** 2 * np.asarray(norms2, dtype=np.float64)) * dt)


def potential_half_phase(v: np.ndarray, gamma: float, dt: float) -> np.ndarray:
    """exp(-i dt v / (2 gamma)): half a potential step (eq. StrangTDSE)."""
    return np.exp(-1j * dt * np.asarray(v, dtype=np.float64) / (2.0 * gamma))


# --------------------------------------------------------------------------
# Strang loop
# --------------------------------------------------------------------------
def strang_step(u: np.ndarray, Ph: np.ndarray, K: np.ndarray, n) -> np.ndarray:
    a = Ph * u
    b = samples(K * coeffs(a, n), n)
    return Ph * b


def strang(u0: np.ndarray, v: np.ndarray, norms2: np.ndarray, n, gamma: float,
           dt: float, nsteps: int) -> np.ndarray:
    """nsteps Strang steps of size dt from u0 (physical samples)."""
    Ph = potential_half_phase(v, gamma, dt)
    K = kinetic_phase(norms2, gamma, dt)
    u = np.asarray(u0, dtype=np.complex128).copy()
    for _ in range(int(nsteps)):
        u = strang_step(u, Ph, K, n)
    return u


# --------------------------------------------------------------------------
# Values computed one at a time (spot checks on lattices too large for the
# full oracle run)
# --------------------------------------------------------------------------
def coeff_at(u: np.ndarray, n, xi: np.ndarray) -> np.ndarray:
    """uhat at the bins xi (rows (xi_1, ..., xi_r)) by the direct sum of eq. approx_uhat.

    With p_k = sum_i z_i k_i / n_i, h . p_k = sum_i xi_i k_i / n_i mod 1
    (xi_i = h . z_i mod n_i), so uhat(xi) = (1/N) sum_k u_k exp(-2 pi i sum_i xi_i k_i / n_i).
    Each exponent is reduced in integers before it is evaluated.  For r = 2
    the sum over k is written as e_1^T U e_2 with e_i[k_i] = exp(-2 pi i xi_i k_i / n_i):
    O(N) per bin, no transform.
    """
    s = _shape(n)
    N = int(np.prod(s))
    U = np.asarray(u, dtype=np.complex128).reshape(s)
    xi = np.atleast_2d(np.asarray(xi, dtype=np.int64))
    out = np.empty(xi.shape[0], dtype=np.complex128)
    for t, row in enumerate(xi):
        es = [np.exp(-2j * np.pi * ((int(row[i]) * np.arange(s[i], dtype=np.int64)) % s[i]) / s[i])
              for i in range(len(s))]
        acc = U
        for e in reversed(es):
            acc = acc @ e
        out[t] = acc / N
    return out


def plane_wave_evolution(xi: np.ndarray, norms2: np.ndarray, c: np.ndarray, n, gamma: float,
                         dt: float, nsteps: int, v_const: float, kappa: np.ndarray) -> np.ndarray:
    """Exact state after nsteps Strang steps for u_0 = sum_j c_j exp(2 pi i h_j . x) and v = v_const.

    A constant potential commutes with the Laplacian, so each Strang step is the
    exact propagator (Sec. 2.4: the splitting error is a commutator): plane wave
    h_j picks up exp(-i dt (v_const / gamma + gamma 2 pi^2 ||h_j||^2)) per step
    (eq. Fourier-ODE for the kinetic part, eq. StrangTDSE for the potential).
    This holds on the lattice when each h_j is the anti-aliasing representative
    of its bin xi_j with norm norms2[j].  Returns u_N at the multi-indices
    kappa (rows (k_1, ..., k_r)), with exp(2 pi i h . p_k) = exp(2 pi i sum_i xi_i k_i / n_i).
    """
    s = _shape(n)
    xi = np.atleast_2d(np.asarray(xi, dtype=np.int64))
    kappa = np.atleast_2d(np.asarray(kappa, dtype=np.int64))
    T = float(nsteps) * float(dt)
    out = np.zeros(kappa.shape[0], dtype=np.complex128)
    for j in range(xi.shape[0]):
        ang = -T * (v_const / gamma + gamma * 2.0 * np.pi ** 2 * float(norms2[j]))
        turns = np.zeros(kappa.shape[0], dtype=np.float64)
        for i in range(len(s)):
            turns += ((int(xi[j, i]) * kappa[:, i]) % s[i]) / s[i]
        out += complex(c[j]) * np.exp(1j * ang) * np.exp(2j * np.pi * turns)
    return out


def strang_composed(u0: np.ndarray, v: np.ndarray, norms2: np.ndarray, n, gamma: float, dt: float,
                    nsteps: int, weights) -> np.ndarray:
    """nsteps steps of S(w_s dt) ... S(w_1 dt): a composition of Strang steps (higher-order
    splitting, named as an extension in Sec. 5); each stage is one strang_step of size w_i dt."""
    tables = [(potential_half_phase(v, gamma, w * dt), kinetic_phase(norms2, gamma, w * dt)) for w in weights]
    u = np.asarray(u0, dtype=np.complex128).copy()
    for _ in range(int(nsteps)):
        for Ph, K in tables:
            u = strang_step(u, Ph, K, n)
    return u


# --------------------------------------------------------------------------
# Observables (Sec. 3.3)
# --------------------------------------------------------------------------
def norm2(u: np.ndarray) -> float:
    """||u_a||_{L2}^2 = (1/N) sum |u_kappa|^2 = sum |uhat_chi|^2 (Parseval on the lattice)."""
    return float(np.mean(np.abs(u) ** 2))


def energy(u: np.ndarray, v: np.ndarray, norms2: np.ndarray, n, gamma: float) -> float:
    """<H u, u> with H = -(gamma/2) Lap + v / gamma (Sec. 3.3)."""
    uh = coeffs(u, n)
    kin = (gamma / 2.0) * np.sum(4.0 * np.pi ** 2 * norms2 * np.abs(uh) ** 2)
    pot = np.mean(np.asarray(v) * np.abs(u) ** 2) / gamma
    return float(kin + pot)


def inner(a: np.ndarray, b: np.ndarray) -> complex:
    """<a, b> = (1/N) sum conj(a_k) b_k (lattice-rule L2 inner product)."""
    return complex(np.mean(np.conj(a) * b))


def overlap_objective(u: np.ndarray, phi: np.ndarray) -> float:
    """J = |<u, phi>|^2."""
    return abs(inner(u, phi)) ** 2


# --------------------------------------------------------------------------
# Adjoint (reverse mode through the Strang loop; not part of the paper)
# --------------------------------------------------------------------------
def strang_adjoint(u0: np.ndarray, v: np.ndarray, norms2: np.ndarray, n, gamma: float,
                   dt: float, nsteps: int, phi: np.ndarray, ckpt: int = 0):
    """J = |<u_N, phi>|^2 and its gradients w.r.t. v (real) and u0 (complex).

    Gradients use the convention g = dJ/dRe + i dJ/dIm.  For y = P o x with
    P = exp(-i a v): dJ/dv_k += a * Im(conj(lam_y,k) * y_k) and lam_x = conj(P) lam_y.
    For the kinetic block b = F^{-1} K F a: lam_a = F^{-1} conj(K) F lam_b.
    States are recomputed per segment from checkpoints every `ckpt` steps.
    Returns (J, grad_v, grad_u0, u_N).
    """
    N = int(nsteps)
    ckpt = ckpt if ckpt > 0 else max(1, int(np.ceil(np.sqrt(max(N, 1)))))
    Ph = potential_half_phase(v, gamma, dt)
    K = kinetic_phase(norms2, gamma, dt)
    alpha = dt / (2.0 * gamma)
    u = np.asarray(u0, dtype=np.complex128).copy()
    checkpoints = {}
    for k in range(N):
        if k % ckpt == 0:
            checkpoints[k] = u.copy()
        u = strang_step(u, Ph, K, n)
    uN = u
    c = inner(phi, uN)                          # <phi, u_N>
    J = abs(c) ** 2
    M = uN.size
    lam = 2.0 * c * np.asarray(phi, dtype=np.complex128) / M
    grad_v = np.zeros(M, dtype=np.float64)
    starts = sorted(checkpoints.keys())
    for s in reversed(starts):
        e = min(s + ckpt, N)
        states = [checkpoints[s]]
        for _ in range(s, e - 1):
            states.append(strang_step(states[-1], Ph, K, n))
        for k in range(e - 1, s - 1, -1):
            x = states[k - s]
            a = Ph * x
            b = samples(K * coeffs(a, n), n)
            y = Ph * b
            grad_v += alpha * np.imag(np.conj(lam) * y)
            lam_b = np.conj(Ph) * lam
            lam_a = samples(np.conj(K) * coeffs(lam_b, n), n)
            grad_v += alpha * np.imag(np.conj(lam_a) * a)
            lam = np.conj(Ph) * lam_a
    return J, grad_v, lam, uN
