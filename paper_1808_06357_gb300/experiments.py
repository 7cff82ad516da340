"""The paper's numerical experiments, run on the GPU through the library.

* Sec. 3.2, convergence in the time step: at t = 1, the error of u^m (m steps of
  size 1/m) against a reference u^M with M = 10000 steps, for g1 / g2 and v1 / v2 on
  the Table 1 lattices; Strang splitting gives second order.
* Sec. 3.3, conservation: the variation delta = (max - min) / mean of the norm and of
  the energy <H u, u> over the run (lsp_observables).
* Sec. 3.4, initial discretisation error e_total of g1 against its exact Fourier
  coefficients (closed form through the Faddeeva function).

Inputs come from the workload module (Table 1 generating vectors, g1, g2, v1, v2 at
the lattice points the library returns); every Strang step runs in the library's
kernels.  Errors are measured on the device in the lattice-rule L2 norm
sqrt((1/n) sum |u - u_ref|^2).

    python -m paper_1808_06357_gb300.experiments convergence --d 2 --log2n 18 --init g1 --pot v2 --gamma 0.5
    python -m paper_1808_06357_gb300.experiments conservation --d 5 --log2n 25 --gamma 0.5
    python -m paper_1808_06357_gb300.experiments initial_error --d 4 --log2n 25 --gamma 1
"""

from __future__ import annotations

import argparse
import json
import math
import os
import sys


def _setup(d, n_log2, init, pot, gamma, prec, device=0):
    import torch

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads as w
    from . import _binding as B

    inst = w.paper_instance(d, n_log2, init=init, pot=pot, gamma=gamma)
    plan = B.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec, device=device)
    pts = plan.lattice_points()
    dev = torch.device("cuda", device)
    v = torch.from_numpy(inst.v(pts)).to(dev)
    u0 = torch.from_numpy(inst.u0(pts)).to(dev)
    del pts
    plan.set_potential(v)
    return plan, u0, inst


def convergence(d=2, n_log2=18, init="g1", pot="v2", gamma=0.5, ms=(5, 10, 20, 50, 100, 200, 500, 1000),
                M=10000, T=1.0, prec="c128", device=0):
    """Errors ||u^M - u^m|| at time T and the observed orders between consecutive m."""
    import torch
    plan, u0, inst = _setup(d, n_log2, init, pot, gamma, prec, device)
    plan.set_state(u0)
    plan.strang_steps(T / M, M)
    ref = plan.get_state(prec="c128")
    errs = {}
    for m in ms:
        plan.set_state(u0)
        plan.strang_steps(T / m, m)
        u = plan.get_state(prec="c128")
        errs[m] = float(torch.sqrt(torch.mean(torch.abs(u - ref) ** 2)))
    if plan.status() != 0:
        raise RuntimeError("device status " + str(plan.status()))
    ms = list(ms)
    orders = {f"{a}->{b}": math.log(errs[a] / errs[b]) / math.log(b / a) for a, b in zip(ms, ms[1:])
              if errs[a] > 0 and errs[b] > 0}
    return {"experiment": "convergence", "lattice": inst.name, "n": inst.npoints, "prec": prec, "T": T, "M": M,
            "errors": errs, "orders": orders}


def conservation(d=5, n_log2=25, init="g1", pot="v2", gamma=0.5, dt=1e-3, T=1.0, every=10, prec="c128", device=0):
    """Norm and energy every `every` steps over [0, T]; delta = (max - min) / mean of each."""
    plan, u0, inst = _setup(d, n_log2, init, pot, gamma, prec, device)
    plan.set_state(u0)
    nsteps = int(round(T / dt))
    norms, energies = [], []
    k = 0
    while True:
        nn, e = plan.observables()
        norms.append(nn)
        energies.append(e)
        if k >= nsteps:
            break
        s = min(every, nsteps - k)
        plan.strang_steps(dt, s)
        k += s

    def delta(x):
        return (max(x) - min(x)) / (sum(x) / len(x))

    return {"experiment": "conservation", "lattice": inst.name, "n": inst.npoints, "prec": prec, "dt": dt, "T": T,
            "samples": len(norms), "delta_norm": delta(norms), "delta_energy": delta(energies),
            "norm": norms, "energy": energies}


# --------------------------------------------------------------------------
# Sec. 3.4: the initial discretisation error of g1
# --------------------------------------------------------------------------
def g1_factor(h, c: float, gamma: float):
    """I(h) = int_0^1 exp(-(2 pi x - c)^2 / gamma) exp(-2 pi i h x) dx, closed form.

    With y = 2 pi x - c and the square completed,
        I(h) = exp(-i h c) / (2 pi) * sqrt(pi gamma) / 2 * [E(y)]_{y=-c}^{2 pi - c},
        E(y) = exp(-gamma h^2 / 4) erf((y + i gamma h / 2) / sqrt(gamma)),
    and E is evaluated through the Faddeeva function w (erf z = 1 - exp(-z^2) w(i z) for
    Re z >= 0, odd symmetry otherwise), so that no factor overflows for large h.
    """
    import numpy as np
    from scipy.special import wofz
    h = np.asarray(h, dtype=np.float64)
    sg = math.sqrt(gamma)
    es = np.exp(-gamma * h * h / 4.0)

    def E(y):
        z = (y + 0.5j * gamma * h) / sg
        tail = np.exp(-y * y / gamma - 1j * h * y)             # exp(-gamma h^2 / 4 - z^2)
        return es - tail * wofz(1j * z) if y >= 0 else -(es - tail * wofz(-1j * z))

    return np.exp(-1j * h * c) / (2.0 * math.pi) * (math.sqrt(math.pi * gamma) / 2.0) * (E(2 * math.pi - c) - E(-c))


def g1_norm_factor(c: float, gamma: float) -> float:
    """int_0^1 exp(-2 (2 pi x - c)^2 / gamma) dx (one factor of ||g1||^2 before normalisation)."""
    from scipy.special import erf
    a = math.sqrt(2.0 / gamma)
    return (1.0 / (2.0 * math.pi)) * math.sqrt(math.pi * gamma / 2.0) / 2.0 * (erf(a * (2 * math.pi - c)) - erf(-a * c))


def g1_centres(d: int):
    return [1.5 * math.pi] + [math.pi] * (d - 1)


def g1_coefficients(H, gamma: float):
    """Exact Fourier coefficients ghat(h) of g1 with unit L2 norm on [0,1)^d, for the rows h of H."""
    import numpy as np
    H = np.asarray(H)
    d = H.shape[1]
    cs = g1_centres(d)
    norm2 = 1.0
    for c in cs:
        norm2 *= g1_norm_factor(c, gamma)
    out = np.full(H.shape[0], 1.0 / math.sqrt(norm2), dtype=np.complex128)
    for j in range(d):
        lo, hi = int(H[:, j].min()), int(H[:, j].max())
        tab = g1_factor(np.arange(lo, hi + 1), cs[j], gamma)
        out *= tab[H[:, j] - lo]
    return out


def initial_error(d=2, n_log2=18, gamma=1.0, prec="c128", device=0):
    """e_total = ||g1 - g1_a||_L2 (Sec. 3.4): with ||g1|| = 1,
    e_total^2 = 1 - sum_{h in A} |ghat(h)|^2 + sum_{h in A} |ghat(h) - ghat_a(h)|^2,
    ghat exact (g1_coefficients), ghat_a the lattice-rule coefficients computed by the library."""
    import numpy as np
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads as w
    from . import _binding as B
    z = w.table1_z(d, n_log2)
    plan = B.Plan(z, (1 << n_log2,), gamma, prec=prec, device=device)
    pts = plan.lattice_points()
    cs = np.array(g1_centres(d))
    shape = np.exp(-np.sum((2.0 * np.pi * pts - cs) ** 2, axis=1) / gamma)
    del pts
    norm2 = 1.0
    for c in cs:
        norm2 *= g1_norm_factor(float(c), gamma)
    plan.set_state(torch.from_numpy((shape / math.sqrt(norm2)).astype(np.complex128)).to(torch.device("cuda", device)))
    ga = plan.get_state(space="spectral", prec="c128").cpu().numpy()
    g = g1_coefficients(plan.index_table(), gamma)
    inside = float(np.sum(np.abs(g) ** 2))
    alias = float(np.sum(np.abs(g - ga) ** 2))
    e2 = max(0.0, 1.0 - inside) + alias
    return {"experiment": "initial_error", "d": d, "n": 1 << n_log2, "gamma": gamma, "prec": prec,
            "outside_A": max(0.0, 1.0 - inside), "aliasing": alias, "e_total": math.sqrt(e2)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("experiment", choices=["convergence", "conservation", "initial_error"])
    ap.add_argument("--d", type=int, default=2)
    ap.add_argument("--log2n", type=int, default=18)
    ap.add_argument("--init", default="g1", choices=["g1", "g2"])
    ap.add_argument("--pot", default="v2", choices=["v1", "v2"])
    ap.add_argument("--gamma", type=float, default=0.5)
    ap.add_argument("--prec", default="c128", choices=["c64", "c128"])
    ap.add_argument("--M", type=int, default=10000)
    ap.add_argument("--ms", default="5,10,20,50,100,200,500,1000")
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--T", type=float, default=1.0)
    ap.add_argument("--every", type=int, default=10)
    a = ap.parse_args(argv)
    if a.experiment == "convergence":
        r = convergence(a.d, a.log2n, a.init, a.pot, a.gamma, tuple(int(x) for x in a.ms.split(",")), a.M, a.T, a.prec)
    elif a.experiment == "initial_error":
        r = initial_error(a.d, a.log2n, a.gamma, a.prec)
    else:
        r = conservation(a.d, a.log2n, a.init, a.pot, a.gamma, a.dt, a.T, a.every, a.prec)
        r = {k: v for k, v in r.items() if k not in ("norm", "energy")}
    print(json.dumps(r))


if __name__ == "__main__":
    main()
