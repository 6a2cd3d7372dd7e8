"""CPU oracle for the nested-dissection NEGF diagonal solver -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import anything from this package.  The product path (the CUDA
library and its Python binding) never imports it, and this package never imports
the product path: the two share no arithmetic.  The one shared module is the
seeded input generator ``paper_1305_1070_gb300.workloads``, which holds no
Green's-function arithmetic.

Everything here is plain numpy/scipy in complex128 (the paper fixes no
precision).  Contents:

* ``leads``      -- surface Green's functions and contact self-energies of
                    semi-infinite leads (closed form per transverse mode, and
                    Lopez-Sancho decimation), paper Sec. 2.
* ``selfenergy`` -- Fermi function, broadening Gamma, lesser/greater
                    self-energies, constant-broadening phonon model.
* ``dense``      -- the definition, Eq. (1)-(2): A = (E + i eta) I - H - Sigma,
                    G^r = A^{-1}, G^< = G^r Sigma^< G^a, G^> = G^r Sigma^> G^a.
* ``rgf``        -- the recursive Green's function method (Sec. 2), exact up to
                    rounding, used where dense inversion is infeasible.
* ``sampled``    -- single diagonal entries by one sparse solve per site
                    (definition, usable at any size).
* ``nd_reference`` -- the paper's multilevel fold/extract algorithm (Sec. 3.2)
                    written out block by block on a cluster tree; a test aid
                    that checks the block algebra, not the parity oracle.
* ``scba``       -- self-consistent Born iteration of an elastic local phonon
                    self-energy (Sigma_ph,jj = D G_jj), densely per energy.
* ``observables`` -- density, terminal current, transmission, error metric.
* ``response``   -- the density with an on-site potential U and its Jacobian
                    dn/dU from the dense definition, and the per-energy terms
                    of the adjoint (c^T dn/dU) and forward ((dn/dU) v) products.
* ``poisson``    -- the five-point Poisson operator of the self-consistent
                    loop (Dirichlet at the transport ends, Neumann at the edges).
* ``sp``         -- Newton iteration of the Schroedinger-Poisson problem with
                    the dense Jacobian.
* ``transfer``   -- 2x2 transfer-matrix transmission of a 1D chain, an
                    independent textbook method used to pin the oracle.
* ``nd_general`` -- the Sec. 3.2 algorithm as a block LU (left and right
                    factors) for a general A, block by block: the form a
                    general-Hermitian kernel path would run; a test aid.
* ``hermitian``  -- the definition for a general Hermitian H (complex
                    hoppings, e.g. a magnetic field), where A is not complex
                    symmetric: conjugate transpositions in the leads and the
                    self-energies; the case the symmetric elimination cannot
                    take.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against
something other than itself (closed forms, brute force, invariants, independent
methods); see ``tests/test_oracle_*.py``.
"""
