"""CPU FP64 oracle for the MIDBF apply — TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never imports,
links or executes anything here, and nothing here imports the product.

What it computes, each function citing the passage of Chen, Zhang, Ho & Yang,
"Multidimensional Phase Recovery and Interpolative Decomposition Butterfly
Factorization" (arXiv 1908.09376) that it follows:

* ``direct``   — the exact matvec of eq. (1) by direct summation, the dense K.
* ``fftcheck`` — closed form of eq. (1) for Phi = x.xi on uniform grids (FFT).
* ``phase``    — the phase functions of the workloads (Example 1 and variants).
* ``tree``     — quad/oct trees with Z-order (Sec. 3.1, Fig. 6; Sec. 3.6).
* ``idec``     — linear-scaling interpolative decompositions (Sec. 3.2).
* ``midbf``    — LRCS (Sec. 3.3), MSCS (Sec. 3.4), recursive MSCS (Sec. 3.5)
                 and the apply of the factor product, eq. (finishIDBF).
* ``planio``   — reader/writer of the level-program file format, so the same
                 factors can be applied here and on the GPU.
* ``recovery`` — Algorithms 1, 4, 5, 6, 7 (Sec. 2.1, 2.3).

Parity status of each function is stated in its module docstring.
"""
