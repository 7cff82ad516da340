"""Seeded synthetic inputs for the lattice Strang-splitting TDSE solver.

This module is shared by the tests, the benchmark and the oracle as the single
source of inputs.  It holds none of the method's arithmetic: it defines input
functions (potentials v, initial states g), generating vectors and run
parameters, and a portable counter-based random generator.  Sampling a
function at lattice points uses the points handed to it by the caller.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here so that every
platform (x86 host, Arm GPU host) draws identical values.

Workloads follow the paper's setting (Sec. 1 TDSE on the d-torus; Sec. 3.2
initial conditions and potentials) and the five hot-path configurations:

  C1  d=2, z=(1,31), n=961, explicit box |h_j|<=15, gamma=0.1,
      v = prod_j (1 - cos 2 pi x_j), Gaussian sigma=0.1 at 0.5 with momentum 3
      along x_1, dt=1e-3, 1000 steps.
  C2  d=6, n=2^22, reconstructing rank-1 lattice for the hyperbolic cross
      prod(1+|h_j|) <= 64, minimal-l2 anti-aliasing set, gamma=0.05,
      v = sum_j cos 2 pi x_j + 0.5 prod_j cos 2 pi x_j, Gaussian sigma=0.08,
      dt=1e-3, 1000 steps.
  C3  256 instances, d in 3..8, n = 2^m with m in 12..20, per-instance dt
      log-uniform in [1e-4, 1e-2], random cosine-series v with |h|^-5 decay,
      gamma=0.1, 500 steps.
  C4  d=4, n=2^20, gamma=0.1, v = prod_j (1 - cos 2 pi x_j), dt=1e-3,
      500 steps, objective |<u_T, phi>|^2 with phi a shifted Gaussian.
  C5  rank-2 lattice, d=16, n=(2^14, 2^12), hyperbolic cross bound 16,
      v = sum_{j<k} 0.1 cos 2 pi (x_j - x_k), product Gaussian, gamma=0.1,
      dt=1e-3, batch 4, 200 steps.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Optional, Sequence

import numpy as np

_MASK = (1 << 64) - 1


# --------------------------------------------------------------------------
# SplitMix64 counter-based generator
# --------------------------------------------------------------------------
def _splitmix64_array(seed: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 output for state = seed + (counter+1) * golden gamma."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + (counters.astype(np.uint64) + np.uint64(1)) * np.uint64(
            0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


class Rng:
    """Deterministic stream of uniforms and integers (SplitMix64)."""

    def __init__(self, seed: int, stream: int = 0):
        self.seed = (int(seed) * 0x2545F4914F6CDD1D + int(stream) * 0x9E3779B97F4A7C15) & _MASK
        self.count = 0

    def u64(self, size: int) -> np.ndarray:
        c = np.arange(self.count, self.count + size, dtype=np.uint64)
        self.count += size
        return _splitmix64_array(self.seed, c)

    def uniform(self, size: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        # 53 high bits -> [0, 1)
        u = (self.u64(size) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
        return lo + (hi - lo) * u

    def integers(self, size: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi) (hi - lo < 2^32), by multiply-shift."""
        span = int(hi - lo)
        r = self.u64(size) >> np.uint64(32)
        return (lo + ((r * np.uint64(span)) >> np.uint64(32)).astype(np.int64)).astype(np.int64)


# --------------------------------------------------------------------------
# Input functions
# --------------------------------------------------------------------------
def periodized_gaussian(x: np.ndarray, center: float, sigma: float) -> np.ndarray:
    """sum_{m in {-1,0,1}} exp(-(x - center + m)^2 / (2 sigma^2)), x in [0,1)."""
    y = x - center
    out = np.zeros_like(y, dtype=np.float64)
    for m in (-1.0, 0.0, 1.0):
        out += np.exp(-((y + m) ** 2) / (2.0 * sigma * sigma))
    return out


def gaussian_packet(points: np.ndarray, sigma: float, centers: Sequence[float],
                    k0: int = 0) -> np.ndarray:
    """prod_j G_sigma(x_j - c_j) * exp(2 pi i k0 x_1), discretely normalised.

    The normalisation makes (1/n) sum_k |u_k|^2 = 1 on the given points, the
    lattice-rule analogue of the unit L2 norm of the paper's initial
    conditions (Sec. 3.2).
    """
    pts = np.asarray(points, dtype=np.float64)
    amp = np.ones(pts.shape[0], dtype=np.float64)
    for j in range(pts.shape[1]):
        amp *= periodized_gaussian(pts[:, j], centers[j], sigma)
    u = amp.astype(np.complex128)
    if k0:
        u = u * np.exp(2j * np.pi * k0 * pts[:, 0])
    nrm = math.sqrt(float(np.mean(np.abs(u) ** 2)))
    return u / nrm


def v_smooth(points: np.ndarray) -> np.ndarray:
    """Paper's smooth potential v_1(x) = prod_j (1 - cos 2 pi x_j) (Sec. 3.2)."""
    pts = np.asarray(points, dtype=np.float64)
    return np.prod(1.0 - np.cos(2.0 * np.pi * pts), axis=1)


def v_harmonic(points: np.ndarray) -> np.ndarray:
    """Paper's harmonic potential v_2(x) = 1/2 sum_j (2 pi x_j - pi)^2 (Sec. 3.2)."""
    pts = np.asarray(points, dtype=np.float64)
    return 0.5 * np.sum((2.0 * np.pi * pts - np.pi) ** 2, axis=1)


def v_cos_sum_prod(points: np.ndarray) -> np.ndarray:
    """sum_j cos 2 pi x_j + 0.5 prod_j cos 2 pi x_j."""
    c = np.cos(2.0 * np.pi * np.asarray(points, dtype=np.float64))
    return c.sum(axis=1) + 0.5 * np.prod(c, axis=1)


def v_pair_cos(points: np.ndarray) -> np.ndarray:
    """sum_{j<k} 0.1 cos 2 pi (x_j - x_k)."""
    pts = np.asarray(points, dtype=np.float64)
    d = pts.shape[1]
    out = np.zeros(pts.shape[0])
    for j in range(d):
        for k in range(j + 1, d):
            out += 0.1 * np.cos(2.0 * np.pi * (pts[:, j] - pts[:, k]))
    return out


@dataclass
class CosSeries:
    """v(x) = sum_t c_t cos(2 pi h_t . x + phi_t): a smooth random potential."""
    h: np.ndarray          # (T, d) integer frequencies
    c: np.ndarray          # (T,)
    phi: np.ndarray        # (T,)

    def __call__(self, points: np.ndarray) -> np.ndarray:
        pts = np.asarray(points, dtype=np.float64)
        out = np.zeros(pts.shape[0])
        for t in range(self.h.shape[0]):
            out += self.c[t] * np.cos(2.0 * np.pi * (pts @ self.h[t].astype(np.float64)) + self.phi[t])
        return out


def random_cos_series(rng: Rng, d: int, terms: int = 16, decay: float = 5.0) -> CosSeries:
    hs = []
    while len(hs) < terms:
        h = rng.integers(d, -2, 3)
        if np.any(h != 0):
            hs.append(h)
    h = np.array(hs, dtype=np.int64)
    c = rng.uniform(terms) * np.linalg.norm(h, axis=1) ** (-decay)
    phi = rng.uniform(terms, 0.0, 2.0 * np.pi)
    return CosSeries(h, c, phi)


# --------------------------------------------------------------------------
# Index sets and generating vectors
# --------------------------------------------------------------------------
def hyperbolic_cross(d: int, bound: int) -> np.ndarray:
    """All h in Z^d with prod_j (1 + |h_j|) <= bound, as an (m, d) int64 array."""
    out = [np.zeros((1, 0), dtype=np.int64)]
    prods = [np.ones(1, dtype=np.int64)]
    cur, cp = out[0], prods[0]
    for _ in range(d):
        rows, ps = [], []
        for a in range(-(bound - 1), bound):
            f = 1 + abs(a)
            keep = cp * f <= bound
            if not np.any(keep):
                continue
            sub = cur[keep]
            rows.append(np.concatenate([sub, np.full((sub.shape[0], 1), a, dtype=np.int64)], axis=1))
            ps.append(cp[keep] * f)
        cur = np.concatenate(rows, axis=0)
        cp = np.concatenate(ps)
    return cur


def box_index_set(d: int, half: int) -> np.ndarray:
    """All h in Z^d with |h_j| <= half (lexicographic, h_1 slowest)."""
    axes = [np.arange(-half, half + 1, dtype=np.int64)] * d
    grids = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.reshape(-1) for g in grids], axis=1)


def _distinct(keys: np.ndarray) -> bool:
    return np.unique(keys).size == keys.size


def reconstructing_rank1(index_set: np.ndarray, n: int, rng: Rng,
                         tries: int = 4000) -> np.ndarray:
    """Seeded component-by-component search for z with h -> h.z mod n injective on I.

    Component 1 is fixed to 1; each later component is drawn uniformly among
    the units mod n (odd numbers when n is a power of two) until the
    projection of I onto the first j coordinates maps injectively.
    """
    I = np.asarray(index_set, dtype=np.int64)
    d = I.shape[1]
    z = [1]
    for j in range(1, d):
        proj = np.unique(I[:, : j + 1], axis=0)
        for _ in range(tries):
            cand = int(rng.integers(1, 1, n)[0])
            if math.gcd(cand, n) != 1:
                continue
            keys = (proj @ np.array(z + [cand], dtype=np.int64)) % n
            if _distinct(keys):
                z.append(cand)
                break
        else:
            raise RuntimeError(f"no injective component {j} found")
    return np.array(z, dtype=np.int64)


def cbc_candidates(d: int, n, count: int, rng: Rng) -> np.ndarray:
    """Seeded candidate lists for a component-by-component search: (d - 1, count, r)
    units modulo each n_i (odd numbers when n_i is a power of two)."""
    nt = [int(x) for x in np.atleast_1d(n)]
    out = np.zeros((d - 1, count, len(nt)), dtype=np.int64)
    for j in range(d - 1):
        for t in range(count):
            for i, ni in enumerate(nt):
                while True:
                    c = int(rng.integers(1, 1, ni)[0])
                    if math.gcd(c, ni) == 1:
                        break
                out[j, t, i] = c
    return out


def reconstructing_rank2(index_set: np.ndarray, n1: int, n2: int, rng: Rng,
                         tries: int = 4000) -> np.ndarray:
    """Seeded search for Z = (z_1, z_2) with h -> (h.z_1 mod n1, h.z_2 mod n2) injective on I.

    Component 0 is fixed to (1, 0) and every later component is (a, b) with a a
    unit mod n1 and b a unit mod n2, so (1, 0) and (0, 1) lie in the image of
    h -> (h.z_1, h.z_2): the map onto Z_n1 x Z_n2 is surjective and the n1 n2
    lattice points are distinct.  (With n1, n2 both even, making every
    component of z_2 a unit as well would confine the image mod 2 to the
    diagonal and merge the points k and k + (n1/2, n2/2).)
    """
    I = np.asarray(index_set, dtype=np.int64)
    d = I.shape[1]
    z1, z2 = [1], [0]
    for j in range(1, d):
        proj = np.unique(I[:, : j + 1], axis=0)
        for _ in range(tries):
            a = int(rng.integers(1, 1, n1)[0])
            b = int(rng.integers(1, 1, n2)[0])
            if math.gcd(a, n1) != 1 or math.gcd(b, n2) != 1:
                continue
            k1 = (proj @ np.array(z1 + [a], dtype=np.int64)) % n1
            k2 = (proj @ np.array(z2 + [b], dtype=np.int64)) % n2
            if _distinct(k1 * n2 + k2):
                z1.append(a)
                z2.append(b)
                break
        else:
            raise RuntimeError(f"no injective component {j} found")
    return np.stack([np.array(z1, dtype=np.int64), np.array(z2, dtype=np.int64)], axis=1)


def random_rank1(d: int, n: int, rng: Rng) -> np.ndarray:
    """Seeded rank-1 generating vector: z_1 = 1, other components random units mod n."""
    z = [1]
    while len(z) < d:
        c = int(rng.integers(1, 1, n)[0])
        if math.gcd(c, n) == 1:
            z.append(c)
    return np.array(z, dtype=np.int64)


# --------------------------------------------------------------------------
# Workload descriptions
# --------------------------------------------------------------------------
def plane_waves(xi: np.ndarray, c: Sequence[complex], n) -> np.ndarray:
    """u_k = sum_j c_j exp(2 pi i sum_i xi_ji k_i / n_i) for every multi-index k (lexicographic).

    This is the sum of the plane waves exp(2 pi i h_j . x) sampled at the
    lattice points, h_j . z_i = xi_ji mod n_i.  Exponents are reduced in
    integers; each term is an outer product of one-dimensional factors.
    """
    s = tuple(int(x) for x in np.atleast_1d(n))
    xi = np.atleast_2d(np.asarray(xi, dtype=np.int64))
    out = np.zeros(s, dtype=np.complex128)
    for j in range(xi.shape[0]):
        term = np.array(complex(c[j]), dtype=np.complex128)
        for i in range(len(s)):
            e = np.exp(2j * np.pi * ((int(xi[j, i]) * np.arange(s[i], dtype=np.int64)) % s[i]) / s[i])
            term = np.multiply.outer(term, e)
        out += term
    return out.reshape(-1)


def c5_fields(inst: "Instance", rows_per_chunk: int = 256):
    """C5's v (v_pair_cos) and u0 (product Gaussian, sigma 0.1 at 0.5) on a rank-2 lattice.

    Evaluated without materialising the (N, d) point array: coordinate j of
    point (k1, k2) is t_j / n1 with t_j = (z1_j k1 + z2_j k2 n1 / n2) mod n1,
    so every one-dimensional factor is a lookup in a table of n1 values, and
    sum_{j<k} cos 2 pi (x_j - x_k) = (|sum_j exp(2 pi i x_j)|^2 - d) / 2.
    Same values as v_pair_cos and gaussian_packet on lattice_points up to
    rounding; the discrete normalisation is the same.
    """
    n1, n2 = int(inst.n[0]), int(inst.n[1])
    Zm = inst.Zmat.astype(np.int64) % np.array([n1, n2], dtype=np.int64)
    d = Zm.shape[0]
    t = np.arange(n1, dtype=np.int64)
    etab = np.exp(2j * np.pi * t / n1)
    gtab = periodized_gaussian(t / n1, 0.5, 0.1)
    step2 = n1 // n2
    k2 = np.arange(n2, dtype=np.int64)
    col = [(Zm[j, 1] * step2 * k2) % n1 for j in range(d)]
    v = np.empty(n1 * n2, dtype=np.float64)
    u = np.empty(n1 * n2, dtype=np.complex128)
    for r0 in range(0, n1, rows_per_chunk):
        k1 = np.arange(r0, min(n1, r0 + rows_per_chunk), dtype=np.int64)
        acc = np.zeros((k1.size, n2), dtype=np.complex128)
        amp = np.ones((k1.size, n2), dtype=np.float64)
        for j in range(d):
            tj = ((Zm[j, 0] * k1) % n1)[:, None] + col[j][None, :]
            tj %= n1
            acc += etab[tj]
            amp *= gtab[tj]
        sl = slice(r0 * n2, (r0 + k1.size) * n2)
        v[sl] = (0.05 * (np.abs(acc) ** 2 - d)).reshape(-1)
        u[sl] = amp.reshape(-1)
    u /= math.sqrt(float(np.mean(np.abs(u) ** 2)))
    return v, u


# --------------------------------------------------------------------------
# The paper's own experiments (Sec. 3.1 Table 1; Sec. 3.2 g1, g2, v1, v2)
# --------------------------------------------------------------------------
# Generating vectors of Table 1 (Sec. 3.1): d = 2 and 3 have their own rows; for
# d = 4..12 the paper uses n = 2^25 and the first d components of the 12-vector.
TABLE1_ROWS = {(2, 18): (1, 100135), (2, 20): (1, 443165), (3, 22): (1, 1737355, 261247),
               (3, 25): (1, 12386359, 15699201)}
TABLE1_Z12 = (1, 12386359, 15699201, 6807287, 13966305, 6107923, 4432603, 2304135, 7323801, 5705679,
              5643703, 3867405)


def table1_z(d: int, n_log2: int) -> np.ndarray:
    if (d, n_log2) in TABLE1_ROWS:
        return np.array(TABLE1_ROWS[(d, n_log2)], dtype=np.int64)
    if 4 <= d <= 12 and n_log2 == 25:
        return np.array(TABLE1_Z12[:d], dtype=np.int64)
    raise ValueError(f"Table 1 has no lattice for d={d}, n=2^{n_log2}")


def _paper_offsets(points: np.ndarray) -> np.ndarray:
    """2 pi x_j - c_j with c_1 = 3 pi / 2 and c_j = pi for j >= 2 (the packet centre of g1, g2)."""
    pts = np.asarray(points, dtype=np.float64)
    c = np.full(pts.shape[1], np.pi)
    c[0] = 1.5 * np.pi
    return 2.0 * np.pi * pts - c


def _unit(u: np.ndarray) -> np.ndarray:
    return u / math.sqrt(float(np.mean(np.abs(u) ** 2)))


def paper_g1(points: np.ndarray, gamma: float) -> np.ndarray:
    """Sec. 3.2 "Gaussian" g1: exp(-sum_j (2 pi x_j - c_j)^2 / gamma), unit lattice-rule norm."""
    y = _paper_offsets(points)
    return _unit(np.exp(-np.sum(y * y, axis=1) / gamma).astype(np.complex128))


def paper_g2(points: np.ndarray, gamma: float) -> np.ndarray:
    """Sec. 3.2 "Hat" g2: prod_j (1 - 2 |2 pi x_j - c_j| / (pi sqrt(gamma))), each factor taken
    as its positive part, unit lattice-rule norm."""
    y = np.abs(_paper_offsets(points))
    f = np.clip(1.0 - 2.0 * y / (np.pi * math.sqrt(gamma)), 0.0, None)
    return _unit(np.prod(f, axis=1).astype(np.complex128))


def paper_instance(d: int, n_log2: int, init: str = "g1", pot: str = "v2", gamma: float = 0.5,
                   dt: float = 1e-3, nsteps: int = 1000) -> Instance:
    """A Sec. 3.2 experiment on a Table 1 lattice: initial condition g1 or g2, potential v1 or v2."""
    z = table1_z(d, n_log2)
    g = paper_g1 if init == "g1" else paper_g2
    return Instance(name=f"paper d={d} n=2^{n_log2} {init} {pot} gamma={gamma}", d=d, n=(1 << n_log2,), Z=z,
                    gamma=gamma, dt=dt, nsteps=nsteps, v=v_smooth if pot == "v1" else v_harmonic,
                    u0=lambda p, _g=g, _gm=gamma: _g(p, _gm))


@dataclass
class Instance:
    """One TDSE problem: lattice, physics parameters and input functions."""
    name: str
    d: int
    n: tuple                       # (n,) rank-1 or (n1, ..., nr)
    Z: np.ndarray                  # (d,) rank-1 or (d, r)
    gamma: float
    dt: float
    nsteps: int
    v: Callable[[np.ndarray], np.ndarray]
    u0: Callable[[np.ndarray], np.ndarray]
    index_set: Optional[np.ndarray] = None   # explicit anti-aliasing set (EXPLICIT mode)
    phi: Optional[Callable[[np.ndarray], np.ndarray]] = None
    extra: dict = field(default_factory=dict)

    @property
    def rank(self) -> int:
        return len(self.n)

    @property
    def npoints(self) -> int:
        return int(np.prod(self.n))

    @property
    def Zmat(self) -> np.ndarray:
        Z = np.asarray(self.Z, dtype=np.int64)
        return Z.reshape(self.d, -1)


def c1() -> Instance:
    d = 2
    return Instance(
        name="C1 d=2 n=961 z=(1,31) box|h|<=15", d=d, n=(961,), Z=np.array([1, 31]),
        gamma=0.1, dt=1e-3, nsteps=1000, v=v_smooth,
        u0=lambda p: gaussian_packet(p, 0.1, [0.5] * d, k0=3),
        index_set=box_index_set(2, 15))


_C2_CACHE = {}


def c2(n_log2: int = 22) -> Instance:
    """C2; below n = 2^22 an HC(64)-injective lattice (51,233 elements) is hard or
    impossible to find, so smaller variants use a seeded random rank-1 lattice."""
    d = 6
    n = 1 << n_log2
    if n_log2 not in _C2_CACHE:
        if n_log2 >= 22:
            _C2_CACHE[n_log2] = reconstructing_rank1(hyperbolic_cross(d, 64), n, Rng(0, 2))
        else:
            _C2_CACHE[n_log2] = random_rank1(d, n, Rng(n_log2, 2))
    z = _C2_CACHE[n_log2]
    return Instance(
        name=f"C2 d=6 n=2^{n_log2} HC(64) reconstructing", d=d, n=(n,), Z=z,
        gamma=0.05, dt=1e-3, nsteps=1000, v=v_cos_sum_prod,
        u0=lambda p: gaussian_packet(p, 0.08, [0.5] * d))


def c3(count: int = 256, seed: int = 0, min_log2: int = 12, max_log2: int = 20) -> list:
    rng = Rng(seed, 3)
    out = []
    for i in range(count):
        d = int(rng.integers(1, 3, 9)[0])
        m = int(rng.integers(1, min_log2, max_log2 + 1)[0])
        n = 1 << m
        dt = float(10.0 ** rng.uniform(1, -4.0, -2.0)[0])
        z = random_rank1(d, n, rng)
        v = random_cos_series(rng, d)
        out.append(Instance(
            name=f"C3[{i}] d={d} n=2^{m}", d=d, n=(n,), Z=z, gamma=0.1, dt=dt, nsteps=500,
            v=v, u0=(lambda dd: (lambda p: gaussian_packet(p, 0.1, [0.5] * dd)))(d)))
    return out


def c4(n_log2: int = 20) -> Instance:
    d = 4
    n = 1 << n_log2
    z = random_rank1(d, n, Rng(0, 4))
    return Instance(
        name=f"C4 d=4 n=2^{n_log2} adjoint", d=d, n=(n,), Z=z, gamma=0.1, dt=1e-3, nsteps=500,
        v=v_smooth, u0=lambda p: gaussian_packet(p, 0.1, [0.5] * d),
        phi=lambda p: gaussian_packet(p, 0.1, [0.6] + [0.5] * (d - 1)))


_C5_CACHE = {}


def c5(n1_log2: int = 14, n2_log2: int = 12, d: int = 16, bound: int = 16) -> Instance:
    n1, n2 = 1 << n1_log2, 1 << n2_log2
    key = (n1_log2, n2_log2, d, bound)
    if key not in _C5_CACHE:
        _C5_CACHE[key] = reconstructing_rank2(hyperbolic_cross(d, bound), n1, n2, Rng(0, 5))
    Z = _C5_CACHE[key]
    return Instance(
        name=f"C5 rank-2 d={d} n=2^{n1_log2}x2^{n2_log2}", d=d, n=(n1, n2), Z=Z, gamma=0.1,
        dt=1e-3, nsteps=200, v=v_pair_cos, u0=lambda p: gaussian_packet(p, 0.1, [0.5] * d),
        extra={"batch": 4})
