"""GB300-native (sm_103a) data-parallel hot path of four-dimensional
tomographic reconstruction by time-domain decomposition (arXiv 1809.09725).

The computation lives in the CUDA library ``libdynrecon.so`` (C ABI in
``include/dynrecon.h``); :mod:`.dynrecon` is its thin binding and
:mod:`.synth` makes seeded synthetic inputs.
"""
from . import dynrecon  # noqa: F401
from .dynrecon import (ADMM_CG, BF16, CHAMBOLLE_POCK, F32, F64, FOURIER, LEGENDRE, DynreconError, Plan,  # noqa: F401
                       admm_solve, dyn_radon_adj, dyn_radon_fwd, solve_params, tv4d_grad, tv4d_grad_adj,
                       tv4d_prox)
