"""Plain, slow FP64 CPU oracle of the RBSOG force step (Chen, Liang & Xu).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call, link or execute anything in this
package.  The CUDA product path (``paper_2501_10946_gb300``) never imports it, and
the two share no code: no kernels, headers, helpers, tables or constant generators.
The only common module is ``paper_2501_10946_gb300.workloads``, which produces seeded
inputs and holds none of the method's arithmetic.

Contents, each restating the paper:
  sog.py        Algorithm 1 (SOG decomposition, C1 smoothness), Eqs. (1), (27)-(38)
  csrc/oracle.c kernel pieces, near field, structure factor, estimators, full-k far field,
                cell list, brute-force lattice sum (Eqs. (33), (50)-(62))
  core.py       ctypes bindings and composite quantities (energies, coefficients)
  philox.py     Philox4x32-10 (Salmon et al. 2011)
  sampler.py    exact i.i.d. draws from P(k) of Eq. (59)
  integrate.py  velocity Verlet and BAOAB Langevin (Algorithm 2, integration step)
  egs.py        the EGS screening of Sec. 1 as two Yukawa kernels, and its envelope
                random-batch estimator, composed from the above by linearity

Every function is pinned by a not-gpu test to something other than itself (printed
table values, closed forms, brute-force sums, exact moments, published test vectors).
"""
