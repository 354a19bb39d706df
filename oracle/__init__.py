"""Plain, slow, obviously correct FP64 CPU oracle of the neural-subspace
reduced-order Newton solve (Sec. 3.1, Eq. 1-2) and of the Lipschitz-loss
training objective (Sec. 4, Eq. 3, 7, 9, 10, 11).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, the smoke check of the build entry
point and the CPU-baseline leg of the benchmark do.  It shares no code with
the CUDA path (no kernels, headers, helpers or constant tables); the only
common code is the seeded input generators in ``workloads``, which hold
none of the method's arithmetic.

Modules
-------
snh       Stable Neo-Hookean energy density, its first and second
          derivatives and the PSD projection used by projective Newton.
fem       rest-shape quantities, lumped mass, per-element energy, gradient
          and (projected) Hessian, and their full-space assembly.
decoder   the MLP subspace map f(z), its forward-mode Jacobian and its
          second-order tangents.
reduced   the reduced objective E(z) of Eq. 2, its gradient and Gauss-Newton
          Hessian, Cholesky + Armijo Newton, implicit Euler stepping.
fullspace full-space projective Newton on Eq. 1 (the reference for the subspace error
          and snapshot generator).
pool      worker processes (spawned, shared memory) that evaluate reduced's
          chunked element sums in parallel; results are added in chunk
          order, so they equal the serial loop's bit for bit.
training  reconstruction loss (Eq. 3), cubature subspace Hessian (Sec. 4.3),
          Lipschitz loss (Eq. 9), combined loss (Eq. 10), Lip estimate
          (Eq. 7), with gradients by float64 autodiff (torch CPU), as the
          paper computes Hessians by autodiff (Sec. 5).

Parity status: every function here is pinned by a test under tests/
(test_oracle_*.py) against closed forms, invariants, finite differences or
brute force; see each module's header.
"""
