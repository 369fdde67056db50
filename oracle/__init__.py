"""Plain FP64 CPU oracle of the single-pass randomized PCA (Yu et al., IJCAI 2017).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import it. The product (the CUDA library and its
Python binding) never calls into it, and it shares no code with the CUDA path.

Modules
-------
philox   Philox4x32-10 counter-based generator and Box-Muller normals, used as the
         paper's ``randn`` for the test matrix Omega (Alg. 4, step 3).
spca     the method itself, step by step in FP64: centering, the one-pass sketch
         loop (Alg. 4 steps 4-8, Eq. 11), the blocked orthonormalisation with
         re-orthogonalisation (Alg. 4 steps 9-16, Eq. 8-10), the SVD of B and the
         truncation (Alg. 4 steps 17-20), the Gram/Cholesky reading of the same
         QB factorisation, Alg. 1 (two passes) and a one-sided Jacobi SVD used as
         a brute-force reference.
"""
