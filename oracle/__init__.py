"""Plain FP64 CPU oracle of the ROM-based BDDC method for level-set lattices.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library imports, links or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

Every function restates a passage of the paper (arXiv 2604.09113) in slow,
readable numpy; each docstring names the section / equation / algorithm it
follows.  Modules:

* ``basis``      GLL-Lagrange and Bernstein bases (Sec. 2.2.2), Gauss rules.
* ``geometry``   level sets, bilinear thresholds, cell maps (Sec. 2.1).
* ``quadrature`` height-function quadrature of trimmed cells (Sec. 2.2.3).
* ``assembly``   pulled-back tensor (Eq. ELA constitutive), full quadrature,
                 fast-assembly tensor I(mu) (Eq. MDEIM I) and Algorithm 4.
* ``rom``        snapshots, SVD basis, magic points (Algorithm 3), GLL
                 interpolation of I_r(mu), MDEIM online (Algorithm 5).
* ``bddc``       DoF classes, Schur complements, coarse DoFs, coarse basis,
                 partition of unity, Algorithms 1-2, PCG, recovery, and the
                 global direct solve of Eq. (BDDC full system).
* ``grad``       compliance and its discrete-adjoint gradient.

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, an invariant, brute force or a library routine, except where a
function's docstring says "parity unpinned".
"""
