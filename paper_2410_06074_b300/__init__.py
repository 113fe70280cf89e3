"""B300-native batched linear-time solve of the Scalable Mechanistic Neural Network layer.

``binding`` is the ctypes view of libsmnn (include/smnn.h); ``api`` adds plan caching
and the ``SmnnSolve`` autograd.Function.  Importing fails loudly if libsmnn.so cannot be
built or loaded: there is no CPU path.
"""
from . import autotune, binding
from .api import HostPipeline, HostStream, SmnnSolve, SolveConfig, get_plan, gradients, smnn_layer, solve
from .binding import ALGO_AUTO, ALGO_CR, ALGO_CR_FUSED, ALGO_SEQ, F32, F32_REFINED, F32_REFINED_DF, F64, Plan, SmnnError

__all__ = ["HostPipeline", "HostStream", "autotune", "binding", "SmnnSolve", "SolveConfig", "get_plan", "gradients", "smnn_layer", "solve",
           "Plan", "SmnnError", "F32", "F32_REFINED", "F32_REFINED_DF", "F64", "ALGO_AUTO", "ALGO_SEQ", "ALGO_CR", "ALGO_CR_FUSED"]
