"""Plain, slow FP64 CPU oracle for CoLA's compositional linear-algebra hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (the CUDA library and its Python binding) never imports,
links or runs anything from here, and nothing here imports the product.

What it computes, each by its plain definition in FP64 (numpy):

* ``linop``   - the operator tree of Sec. 3.1-3.2 (Dense, Diagonal, LowRank,
                Sum, Product, Kronecker, KroneckerSum), MVM by definition,
                dense form by MVM(e_i), transpose rules and Diag rules of
                App. A, leaf enumeration (the flattened parameter tree of
                App. B.2) and the operator derivative in a leaf direction.
* ``krylov``  - (preconditioned) conjugate gradients (Table 5 base case for
                PSD solves), Lanczos with full reorthogonalisation, the
                Householder Arnoldi iteration (Algorithm 2), Gauss quadrature
                on the Lanczos tridiagonal and stochastic Lanczos quadrature
                for log det = Tr(log A) (App. A.2 derived functions, Table 5).
* ``exact``   - closed forms that the iterative results must reach: the
                Kronecker eigendecomposition rules (App. A.1.2) for solves and
                log-determinants of Kronecker products and sums plus s I, the
                product-splitting solve (Sec. 3.2), dense Cholesky / LU
                references, and the exact GP objective and its gradient.
* ``stochastic`` - Hutchinson and doubly stochastic diagonal / trace
                estimators (Sec. 3.3, App. B.1) on given probes, and the
                Rademacher variance of z^T B z.
* ``grad``    - parameter gradients w^T dy/dtheta = -(A^-1 w)^T (dA/dtheta)(A^-1 b)
                (App. B.2, rule 1) and the log-det gradient Tr(A^-1 dA/dtheta)
                (rule 4), both by definition (brute force over leaf entries)
                and in contracted form.
* ``plan``    - the batched launch's integer tile table by its definition.
* ``rng``     - the SplitMix64 counter generator and Rademacher probes that
                seeded SLQ draws (its own implementation from the published
                definition).

Pins (tests/test_oracle_pins.py): brute-force Kronecker products, both vec
identities, eigenvalue products (App. A.1.2), closed-form Dirichlet Laplacian
eigenpairs, Woodbury, Diag rules vs e_i^T A e_i, transpose inner-product
identity, CG vs dense LU, exact log-det vs dense Cholesky, Gauss quadrature
exactness on polynomials, SLQ z-score, gradient vs finite differences,
SplitMix64's published first outputs, PCG with an exact preconditioner (one
step) and against the condition-number bound, Kronecker-sum solves vs dense LU
and the Laplacian spectrum, the order of a product split, Householder
Arnoldi's orthogonality / Arnoldi relation / agreement with Lanczos, and the
estimators' exactness over the full sign hypercube, variance by enumeration
and sampled variances.  No function here is parity-unpinned.
"""
from . import linop, krylov, exact, grad, plan, rng, stochastic  # noqa: F401
