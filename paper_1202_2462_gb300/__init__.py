"""GB300 SAP-multilevel solver for the clover-improved Wilson-Dirac equation.

Frommer, Kahl, Krieg, Leder, Rottmann, "Aggregation-based Multilevel Methods
for Lattice QCD" (Lattice 2011): red-black Schwarz (SAP) smoothing over 4^4
blocks with local minimal-residual block solves, aggregation-based
interpolation with a Galerkin coarse operator, bootstrap set-up, and an outer
flexible GMRES.  The compute path is the C-ABI library libsapmg.so (hand-written
sm_103a CUDA); this package is its Python binding plus a torch convenience
wrapper.  PyTorch supplies device memory and streams only.
"""

from . import binding
from .binding import (
    MG_OK, MG_NOT_CONVERGED, MG_ERR_ARG, MG_ERR_NONFINITE, MG_ERR_OOM, MG_ERR_CUDA, MG_ERR_TIMEOUT,
    MG_ERR_STATE, MG_FP64, MG_FP32, MG_FP16, MG_BF16, MG_BLOCKED, MG_DAGGER, MG_FP64_ON_FP32, PRECISIONS, MgParams, MgSolveInfo,
    MgError, mg_default_params, mg_setup, mg_save, mg_setup_load, dirac_apply, sap_smooth, mg_solve, mg_cgn_solve, mg_harmonic_ritz, mg_eigh, mg_destroy, mg_pack_spinor,
    mg_unpack_spinor, mg_clover_export, mg_get_vectors, mg_get_coarse_op, mg_restrict, mg_prolong,
    mg_coarse_apply, mg_coarse_apply_batch, mg_restrict_batch, mg_prolong_batch, mg_coarse_solve, mg_coarse_solve_noalloc, mg_precondition, mg_set_profiling, mg_get_profile, mg_get_profile_bytes, mg_reset_profile,
    mg_launch_count, mg_probe_peaks, mg_sync, mg_set_wait_limit, mg_get_tuning, mg_get_history, profile_mask, PROFILE_FAMILIES, mg_net_layer_forward, mg_net_layer_forward_bf16, mg_net_layer_backward,
    mg_net_gate_forward, mg_net_gate_backward, mg_net_loss, mg_adam_step,
)
from .solver import Solver

__all__ = [name for name in dir() if not name.startswith("_")]
