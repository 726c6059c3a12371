"""GB300-native entropic optimal transport: log-domain Sinkhorn and SK-NR(l).

The compute path is the CUDA library ``_lib/libeot.so`` (sources in ``csrc/``,
C ABI in ``include/eot.h``); this package only marshals arguments to it
(``eot.py``).  Build the library with ``build.build()`` (nvcc, sm_103a).
"""
from . import eot  # noqa: F401
from .eot import (  # noqa: F401
    EOT_OK, EOT_NOT_CONVERGED, EOT_PENDING, EOT_EINVAL, EOT_ENOMEM, EOT_ENUMERIC,
    EOT_ETIMEDOUT, EOT_ECUDA, EOT_ENOTFOUND, EOT_MEM_HOST, EOT_MEM_DEVICE, EOT_PREC_FP64,
    EOT_PREC_FP32, EOT_PREC_SPLIT_TC, EOT_HESS_DIAG_ALPHA, EOT_HESS_EXACT, EOT_SIDE_COL,
    EOT_SIDE_ROW, Server, default_options, eot_cost, eot_ctransform, eot_kapply,
    eot_ctransform_noalloc, eot_exp2, eot_marginal_error, eot_plan, eot_solve, eot_solve_batch,
    eot_solve_traced, TRACE_DTYPE, eot_batch_tuning,
    eot_spectral_modes, eot_spectral_modes_filtered, eot_batch_plan, eot_sknr_step, eot_server_simulate,
    last_error, load,
    make_problem, solve,
)

__version__ = "0.1.0"
