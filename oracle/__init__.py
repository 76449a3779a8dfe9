"""CPU FP64 oracle for the adaptive-precision HODLR method (Carson, Chen, Liu,
"Mixed Precision HODLR Matrices", arXiv 2407.21637).

This package is TEST INFRASTRUCTURE.  Only the test suite, the smoke check and
the benchmark's CPU-baseline leg may import it.  The GPU library never calls
it, and it never calls the GPU library: the two share no code.  Inputs come
from the separate ``synth`` module.

Plain, slow and written to be checked by eye against the paper:

* ``formats``  Table 1.1 unit roundoffs and round-to-nearest-even emulators
               written from the IEEE-754 / OCP-FP8 format definitions.
* ``tree``     the cluster tree of Def. 2.1 with the ceil-half split of Sect. 4.
* ``kernels``  dense kernel-matrix entries (eq. (4.1) and the synthetic
               workloads).
* ``compress`` truncated-SVD compression of the off-diagonal blocks (Def. 2.3,
               eq. (3.1)) and the adaptive precision rule (Algorithm 3.2).
* ``matvec``   HODLR_MATVEC (Algorithm 3.3) and the dense assembly of H-hat.
* ``bounds``   gamma_n and the error bounds of Thm 3.1, eq. (3.5), Thm 3.5.
* ``lu``       HODLR_LU (Algorithm 3.4) and the triangular solves.
* ``mlp``      the block-rank predictor that sizes the construction's first
               sketch (affine + relu layers, chain-rule gradient, Adam); the
               paper has no learned component, these are plain definitions.

Parity status per function is stated in each module header.
"""
