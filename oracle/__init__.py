"""FP64 CPU oracle for the energy-parallel NEGF hot path of ELEQTRONeX (arXiv 2407.14633).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import or execute it. It shares no code with the CUDA path
(no kernels, headers, helpers, tables or pre/post-processing); the only inputs both
sides see come from the seeded generators in ``paper_2407_14633_gb300/synth.py``,
which hold none of the method's arithmetic.

Everything here is plain numpy in float64 / complex128, written for a reader who checks
it against the paper by eye:

* ``quadrature`` -- Gauss-Legendre nodes (Newton iteration on P_n), the Fermi function,
  the real-axis bias window and the equilibrium complex contour (Sec. 2.2.1, Eq. Rho).
* ``model``      -- block-tridiagonal tight-binding chains for (n,0) zigzag nanotubes in
  mode space and real space, and the semi-infinite leads (Sec. 2.2.1-2.2.2, Sec. 3.1).
* ``leads``      -- surface Green's functions: closed-form root of the dimerised chain
  and Lopez-Sancho/Rubio decimation (Sec. 2.2.2), and Sigma / Gamma (Eq. GR).
* ``green``      -- dense inversion of (E+i eta)I - H - Sigma for tiny systems and the
  block recursion of Alg. 1 / Alg. 2 (read as the textbook left/right-connected RGF).
* ``charge``     -- Fermi-weighted quadrature to per-ring electron count, T(E) and the
  Landauer current (Eq. Rho, Eq. deviceCharacteristics).
* ``selfconsistent`` -- Broyden's modified second method (Alg. 3), the 1D
  finite-difference Poisson stand-in with gate coupling (Thomas algorithm), and the
  self-consistent loop.

Parity status of every function is stated in its docstring; all are pinned by
``tests/test_oracle_*.py`` against closed forms, invariants, brute force or the paper's
printed values (``tests/golden/``).
"""
