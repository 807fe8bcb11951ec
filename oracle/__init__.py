"""CPU FP64 oracle for the MLMC integrated-density-of-states path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
GPU product path (``paper_1611_09784_gb300``) never imports it and shares no
code, table or helper with it; the only module both sides read is
``synthetic`` (seeds, sizes and workload parameters, none of the method's
arithmetic).

Everything here is plain NumPy/SciPy in float64 / complex128, written from the
paper (Plechac & von Schwerin, "Multi-level Monte Carlo acceleration of
computations on multi-layer materials with random defects"):

* ``philox``      counter-based generator (Salmon et al., SC'11) used to draw
                  the vacancy pattern of Sec. 3.2;
* ``lattice``     honeycomb geometry, supercell indexing, Monkhorst-Pack grid
                  (Sec. 3.1, Sec. 4.2);
* ``hamiltonian`` Bloch Hamiltonian H(k) of eq. (3.2a)-(3.2b) with vacancies
                  (Sec. 3.2), nearest neighbours found by brute-force distance;
* ``idos``        smoothed IDoS of eq. (4.1)-(4.2) from ``numpy.linalg.eigvalsh``;
* ``mlmc``        control-variate coupling of Sec. 3.3 and the estimators of
                  Sec. 2 (eqs. (2.2), (2.6), (2.7));
* ``jacobi``      a cyclic Jacobi eigenvalue solver, an independent cross-check
                  of LAPACK for small Hermitian matrices;
* ``tmdc``        the 11-orbital TMDC-shaped model with chalcogen-pair vacancies
                  (Sec. 3.1-3.2, parameters drawn from the generator).

Parity status of every function is stated in its module docstring.
"""
