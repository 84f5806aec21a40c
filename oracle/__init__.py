"""Plain, slow FP64 CPU oracle of the Harmonic Decomposition Factorization (HDF).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (the CUDA library and its Python binding) never calls it, and it
shares no code, tables or constants with that path.

Every function cites the passage of Ryan & Damle, "Linear Time Kernel Matrix
Approximation via Hyperspherical Harmonics" (ICML 2022) that it follows:

* ``kernels``    -- the isotropic kernels of Sec. 4.1 and their derivatives.
* ``chebyshev``  -- Eq. (chebtrunc), the DCT coefficients, the degree choice (Remark 3),
                    and the monomial coefficients t_{i,j} of Eq. (chebdef).
* ``gegenbauer`` -- the Gegenbauer algebra of App. A (A_{ki}), the addition-theorem
                    normaliser Z_k of Eq. (additiontheorem), norms and sphere areas.
* ``harmonics``  -- the index set H_k and real hyperspherical harmonics, evaluated
                    through hyperspherical angles (Eq. additiontheorem, App. B).
* ``radial``     -- the radial functions r^(k) of Eq. (rdef): the literal route
                    (App. A's closed form of T', in mpmath) and the stable route
                    (Gegenbauer projection, the Legendre/Chebyshev-basis fix of Sec. 3.7).
* ``hdf``        -- Algorithm 1 in its symmetric form (Remark 1): scaling, expansion,
                    QR, eigendecomposition, truncation, U and S, then matvec, solve,
                    the frozen-structure adjoint and the dense checker.
* ``cross``      -- Algorithm 1 in its general form for two sets, K(X, Y) ~= U S V^T:
                    joint scaling, two QRs per parity, SVD, truncation, both factors.
* ``krr``        -- kernel ridge regression of Sec. 4.2: k-means blocks, HDF diagonal
                    blocks with exact off-diagonal blocks, the block preconditioner, PCG.

Functions that have no independent pin are marked "parity unpinned" in their docstring.
At present every function used by the parity tests is pinned (see tests/test_oracle_*.py).
"""
