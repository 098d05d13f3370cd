"""CPU oracle for the CTMRG hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import or run anything in this
package.  The library under ``paper_2112_13184_gb300`` never calls it and
shares no code with it.

* ``ctmrg_ref`` -- plain FP64 directional CTMRG on an iTPS unit cell with the
  QR-free projectors (Sec. 2.2), computed from their definition: dense
  half-system matrices and a full LAPACK SVD; reduced density matrices and
  expectation values (Sec. 5.3).
* ``exact`` -- closed forms the oracle is pinned to: Onsager's free energy,
  internal energy and the Onsager-Yang spontaneous magnetisation of the 2D
  Ising model, product-state expectation values.
* ``elements`` -- the operator element format of Sec. 5.2.

Every function here is pinned by a ``-m "not gpu"`` test against something
other than itself (brute-force loops, closed forms, invariants).
"""
