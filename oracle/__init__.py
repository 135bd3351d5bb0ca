"""FP64 CPU oracle for Multi-level Sketched Preconditioning (MSP).

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, step-by-step FP64
restatement of the method of Derezinski, Musco and Yang, "Faster Linear Systems
and Matrix Norm Approximation via Multi-level Sketched Preconditioning"
(arXiv 2405.05865). It exists to check the CUDA path; only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it. The product path (``paper_2405_05865_gb300``) never imports, links or runs
anything here, and this package imports nothing from the product.

Modules
-------
``prng``      counter-based SplitMix64 draws and Floyd sampling (Definition 2.1)
``sketch``    the sparse embedding S (Def 2.1), the level-2 embedding Phi
              (Lemma 2.2), C = A S^T, W = S C, C~ = Phi C (Algorithm 1)
``nystrom``   lambda~, M2 = C~^T C~ + lambda~ W and its factor (Algorithm 1),
              the Woodbury form of M^{-1} (Eq. M_inverse, Section 4.3)
``krylov``    preconditioned Lanczos (Algorithm 6), symmetric preconditioned
              Lanczos (Algorithm 7), PCG and flexible PCG
``msp``       Algorithm 1 + Algorithm 2 (SolveM1), FP64 iterative refinement
``reference`` definition oracles: dense Cholesky x* = (A + lam I)^{-1} b,
              backward error, effective dimension, Schatten-p closed forms
``hutchinson`` Hutchinson trace estimate of tr(A) = |A|_1 for PSD A
``adjoint``   gradients of L = g^T x, x = (K_theta + lam I)^{-1} b
``batch``     batches of instances with several right-hand sides each: the
              definition (independent per-column solves) as a loop
``effdim``    effective dimension d_lambda by Hutchinson over regularised solves,
              and the sketch size / shift rule built on it (Lemma 2.1)
``general``   three-level MSP for (A^T A + lam I) x = c, A rectangular:
              Algorithm 3 with SolveM1 (Algorithm 4) and SolveM2 (Algorithm 5)
``lsq``       least squares by sketch-and-precondition with MSP inner solves
              (the least-squares corollary of Section 3)
``schatten``  Schatten-p, p in (0, 2), from ridge solves through Balakrishnan's
              integral representation (Section 3.2's black-box requirement)
"""
