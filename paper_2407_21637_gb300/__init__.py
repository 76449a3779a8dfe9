"""GB300-native adaptive-precision HODLR matrices (Carson, Chen, Liu,
"Mixed Precision HODLR Matrices", arXiv 2407.21637).

The compute path is libhodlr.so (hand-written sm_103a CUDA behind the C ABI in
include/hodlr.h); this package only marshals arguments.  PyTorch provides
device memory and streams.
"""
from ._lib import PREC, PREC_NAME, HodlrError, load  # noqa: F401
from .hodlr import (HodlrBatch, HodlrMatrix, HodlrPart, RankPredictor, dense_kernel_matvec,  # noqa: F401
                    tree_order)
