"""FP64 CPU oracle for the lattice Strang-splitting TDSE step.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check in
``__graft_entry__.smoke`` and the CPU-baseline / reference arm of ``bench.py``
may import this package.  The product library under
``paper_1808_06357_gb300`` never imports it and shares no code with it.

The oracle is a plain, slow, obviously-correct restatement of what the paper
(Suzuki, Suryanarayana, Nuyens, arXiv:1808.06357) computes:

* ``oracle.lattice`` -- rank-1 and rank-r lattice points (Sec. 2.1, Def. 1),
  the bin map h -> Z^T h mod n (Thm 1(iii)), the dual lattice and character
  property (eqs. dual, char), anti-aliasing sets (Def. 2) and the minimal-l2
  representative per bin (Lemma 4, eq. hrepresenter), both by the paper's
  enumerate-sort-greedy recipe (Sec. 3.1) and by an exact min-plus dynamic
  programme over residues; and a component-by-component search for a lattice
  that maps a given index set injectively (Sec. 3.1's CBC construction with
  Def. 2's injectivity as the acceptance test), pinned by pure-Python pair
  searches and the regular grid's mixed-radix generating vector.
* ``oracle.strang`` -- lattice-rule coefficients (eq. approx_uhat), the
  Strang step of eq. StrangTDSE / Algorithm 1 in physical form, the norm,
  energy and overlap observables (Sec. 3.3), the adjoint gradient of
  |<u_T, phi>|^2, and the dense semi-discrete propagator of eq. ode.
* ``oracle.initial_error`` -- the exact Fourier coefficients of the paper's
  initial function g1 (closed form through the Faddeeva function) and the
  initial discretisation error e_total of Sec. 3.4.

Everything runs in IEEE double precision with numpy; numpy.fft is used as the
FFT primitive.  Parity pins (what fixes each function independently of
itself) are the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.  The
adjoint gradient is not in the paper; it is pinned by central finite
differences of the oracle's own forward map.
"""

from . import initial_error, lattice, strang  # noqa: F401
