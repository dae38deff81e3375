"""Plain FP64 CPU oracle for Tensor Network Monte Carlo (TNMC) on the 2D +-J random-bond
Ising model with open boundaries (arXiv 2409.06538).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA
library (``paper_2409_06538_gb300``) and never imports it.

Each step follows the paper's definitions in its order and notation, with numpy's
QR / SVD as library steps:

* ``philox``        counter-based generator (Salmon et al., SC'11), the one source of
                    random numbers the method draws.
* ``lattice``       Eq. (E) energy, the P(J) bond distribution, the Nishimori line.
* ``boundary_mps``  Sec. II.B: the partition-function network contracted row by row,
                    the bond dimension cut back to D by SVD, every row environment cached.
* ``sampler``       Sec. II.A/II.B: Eq. (Bayes)/(approximate_bayes) conditionals
                    evaluated in reverse contraction order with fixed spins as fields.
* ``metropolis``    Eq. (accptanceratio) and the independence-sampler form of App. A.
* ``observables``   Sec. III.C: energy, magnetisation, two-replica overlap, Binder ratios.
* ``periodic``      Sec. IV: periodic boundaries by a pinned pair of lines per step, the
                    rest of the torus sampled as an open region with the fixed spins as fields.
* ``brute``         exhaustive enumeration used to pin all of the above on small lattices.

Parity status: every function is pinned by the ``-m "not gpu"`` tests in ``tests/``
(brute-force enumeration, closed forms of App. A, Nishimori identities, Philox
known-answer vectors).  No function here is "parity unpinned".
"""
