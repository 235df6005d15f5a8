"""CPU oracle for the SPD-HSS preconditioner of an SPD H^2 matrix (Xing, Huang, Chow).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package: only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.

The oracle is a plain, slow, FP64 numpy/scipy restatement of what the paper computes:

* ``tree``     cluster tree, padding of shallow leaves, admissibility lists (Sec. 2, Sec. 5.1),
               and its expansion to three unknowns per point for the RPY tensor
* ``kernels``  kernel functions, including the RPY tensor, and the dense shifted kernel
               matrix (Sec. 6)
* ``linalg``   column-pivoted Householder QR (Alg. 5.1, step 3)
* ``h2``       proxy-point H^2 representation by interpolative decomposition (Sec. 5.1, Sec. 6)
* ``spdhss``   the quadratic scaling-and-compression construction (Sec. 4, Alg. 4.1) with
               the Lambda-sketch bases of Sec. 5.2.1, on a dense matrix; its tolerance-driven
               form with a growing sketch; and Alg. 4.1 with deterministic (truncated SVD)
               bases, to measure what the sketch costs
* ``ulv``      ULV factorization and solve of a symmetric HSS matrix, and dense solves
* ``pcg``      preconditioned conjugate gradients (Sec. 6.2)

It shares no code with the CUDA path; both only read inputs from
``paper_2011_07632_gb300.inputs`` (seeded random draws, none of the method's arithmetic).
"""
