"""CPU oracle for the mixed dense-sparse interior-point Newton step.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import this package.
The GPU library never calls it, and it never calls the GPU library.

Plain, slow FP64 numpy/scipy code written from the paper's equations:

* `model`     evaluates the synthetic MDS problem of Section 2 (Eqs. (obj)-(bounds)).
* `bk`        Bunch-Kaufman LDL^T (the pivoting of [bunchkaufman] as used by the
              paper's dense solver, Section 2.3), with inertia read from D.
* `kkt`       the 4x4 KKT matrix of Eq. (linsys4x4), its inertia and solve; the
              compressed 3x3 matrix of Eq. (compressed) (path P1); the two-stage
              elimination (path P2); Haynsworth inertia additivity (Section 2.3).
* `ipm`       the filter line-search interior-point loop of Section 2.1
              (Waechter-Biegler), forming and factoring the full KKT matrix.

Pins (tests/test_oracle_*.py, run with -m "not gpu"): brute-force solves and
eigenvalues on tiny inputs, the library LDL^T, closed-form optima of convex
quadratic instances.  See each module's header for the pin of each function.
"""
