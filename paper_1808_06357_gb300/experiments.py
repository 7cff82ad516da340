"""The paper's numerical experiments, run on the GPU through the library.

* Sec. 3.2, convergence in the time step: at t = 1, the error of u^m (m steps of
  size 1/m) against a reference u^M with M = 10000 steps, for g1 / g2 and v1 / v2 on
  the Table 1 lattices; Strang splitting gives second order.
* Sec. 3.3, conservation: the variation delta = (max - min) / mean of the norm and of
  the energy <H u, u> over the run (lsp_observables).
* Sec. 3.4, the lattice-rule coefficients of an initial function (the discrete side of
  its initial discretisation error e_total; the exact coefficients are the caller's).

Inputs are passed in by the caller (a workload instance: Table 1 generating vector,
g1 / g2 and v1 / v2 as functions of the lattice points the library returns); every
Strang step runs in the library's kernels.  Errors are measured on the device in the lattice-rule L2 norm
sqrt((1/n) sum |u - u_ref|^2).

    python -m paper_1808_06357_gb300.experiments convergence --d 2 --log2n 18 --init g1 --pot v2 --gamma 0.5
    python -m paper_1808_06357_gb300.experiments conservation --d 5 --log2n 25 --gamma 0.5
"""

from __future__ import annotations

import argparse
import json
import math


def _setup(inst, prec, device=0):
    import torch

    from . import _binding as B

    plan = B.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec, device=device)
    pts = plan.lattice_points()
    dev = torch.device("cuda", device)
    v = torch.from_numpy(inst.v(pts)).to(dev)
    u0 = torch.from_numpy(inst.u0(pts)).to(dev)
    del pts
    plan.set_potential(v)
    return plan, u0


def convergence(inst, ms=(5, 10, 20, 50, 100, 200, 500, 1000), M=10000, T=1.0, prec="c128", device=0):
    """Errors ||u^M - u^m|| at time T and the observed orders between consecutive m.

    inst: a workload instance (generating vector, n, gamma, v and u0 as functions of the
    lattice points), e.g. workloads.paper_instance(d, log2 n, init, pot, gamma)."""
    import torch
    plan, u0 = _setup(inst, prec, device)
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


def conservation(inst, dt=1e-3, T=1.0, every=10, prec="c128", device=0):
    """Norm and energy every `every` steps over [0, T]; delta = (max - min) / mean of each
    (inst as for convergence)."""
    plan, u0 = _setup(inst, prec, device)
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


def lattice_rule_coefficients(z, n_log2, samples, gamma=1.0, prec="c128", device=0):
    """Sec. 3.4's discrete side: the lattice-rule coefficients ghat_a(h_chi) (eq. approx_uhat)
    of a function given by its samples at the lattice points, with the minimal-l2
    representative h_chi of every bin.

    samples: a callable mapping the (n, d) lattice points to the n complex samples.
    Returns (ghat_a, H): ghat_a in bin order (numpy complex128) and H (n, d) int32.
    e_total = ||g - g_a|| then follows from the exact coefficients of g:
    e_total^2 = ||g||^2 - sum_{h in A} |ghat(h)|^2 + sum_{h in A} |ghat(h) - ghat_a(h)|^2."""
    import numpy as np
    import torch
    from . import _binding as B
    plan = B.Plan(z, (1 << n_log2,), gamma, prec=prec, device=device)
    pts = plan.lattice_points()
    u = np.asarray(samples(pts), dtype=np.complex128)
    del pts
    plan.set_state(torch.from_numpy(u).to(torch.device("cuda", device)))
    ga = plan.get_state(space="spectral", prec="c128").cpu().numpy()
    H = plan.index_table()
    plan.destroy()
    return ga, H


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("experiment", choices=["convergence", "conservation"])
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
    try:
        import workloads as w
    except ImportError as e:
        raise SystemExit("run from the repository root: the input generators (workloads/) are needed") from e
    inst = w.paper_instance(a.d, a.log2n, init=a.init, pot=a.pot, gamma=a.gamma)
    if a.experiment == "convergence":
        r = convergence(inst, tuple(int(x) for x in a.ms.split(",")), a.M, a.T, a.prec)
    else:
        r = conservation(inst, a.dt, a.T, a.every, a.prec)
        r = {k: v for k, v in r.items() if k not in ("norm", "energy")}
    print(json.dumps(r))


if __name__ == "__main__":
    main()
