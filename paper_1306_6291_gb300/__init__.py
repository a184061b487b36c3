"""GB300-native batched closed-form diagonalization of real symmetric 2x2 / 3x3 matrices
(Kronenburg, arXiv:1306.6291): a CUDA library with a C-ABI (include/kdiag.h) and this thin
Python binding. See ``kdiag`` for the entry points."""
from . import kdiag
from .kdiag import (Eig2Fn, Eig3Fn, KdError, StLossFn, eig2, eig2_adjoint, eig3, eig3_adjoint, make_opts,
                    st_loss_bwd, st_loss_fwd)

__all__ = ["kdiag", "eig3", "eig2", "eig3_adjoint", "eig2_adjoint", "st_loss_fwd", "st_loss_bwd", "Eig3Fn",
           "Eig2Fn", "StLossFn", "make_opts", "KdError"]
