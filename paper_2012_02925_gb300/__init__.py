"""GB300-native explicit finite-volume Euler residual and RK stage.

Python face of the C-ABI library ``libfvgb.so`` (``include/fvgb.h``): the
multi-block structured-grid residual (MUSCL + limiter + Roe, Section 2 and
Eq. (flux) of arXiv 2012.02925), the ghost exchange between connected blocks
and the explicit M-step Runge-Kutta stage, on one GPU.  Torch supplies device
memory and streams; every numerical step runs in the library's CUDA kernels.
"""
from ._binding import (EXPORTS, FV_ERR_CUDA, FV_ERR_INVALID_ARG, FV_ERR_NONFINITE, FV_ERR_OOM,
                       FV_ERR_TIMEOUT, FV_ERR_UNSUPPORTED, FV_OK, LIB_PATH, PREC_DF64, PREC_FP32FLUX,
                       PREC_FP64, PRECISIONS, FvError, Solver, load_library, probe_alu_rates)

__all__ = ["Solver", "FvError", "load_library", "probe_alu_rates", "LIB_PATH", "EXPORTS", "PRECISIONS", "PREC_FP64", "PREC_DF64",
           "PREC_FP32FLUX", "FV_OK", "FV_ERR_INVALID_ARG", "FV_ERR_CUDA", "FV_ERR_OOM", "FV_ERR_NONFINITE",
           "FV_ERR_TIMEOUT", "FV_ERR_UNSUPPORTED"]
