"""FP64 CPU oracle for the preconditioned primal-dual method (PDRQS1, Alg. 4) of
"TV-regularized CT Reconstruction and Metal Artifact Reduction Using Inequality
Constraints with Preconditioning" (C. Schiffer, 2018).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library (``paper_1810_03275_gb300``): the Radon pair is plain C
(``radon_ref.c``), everything else is plain numpy in FP64, written step by step
from the thesis.

Parity status of each function is stated in its docstring; all are pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""
from .radon import Geometry, rh_forward, rh_adjoint, rh_forward_entries, rh_adjoint_entries, build_oracle, num_threads
from .pdrq_ref import (
    grad,
    div,
    tv_norm,
    lap_symbol,
    freq_norm,
    precond_symbol,
    precond_symbol_nonneg,
    precond_symbol_from,
    impulse_response_kernel_dft,
    precond_apply,
    flatten,
    unflatten,
    circulant_first_column,
    circulant_kernel_dft,
    circulant_laplace_dft,
    precond_symbol_circulant,
    precond_apply_circulant,
    richardson_m,
    prox_dual,
    tv_project,
    conj_data_term,
    make_descriptors,
    ramlak_kernel,
    ramp_filter,
    fbp,
    dilate_disk,
    metal_trace_estimate,
    power_beta,
    power_c,
    power_start,
    PDRQState,
    pdrq5_solve,
    pdrq2_solve,
    ADMMState,
    pcg,
    soft_threshold2,
    admm_solve,
    pdrq_solve,
    cp_solve,
    diagnostics,
    pdrq_grad,
)

__all__ = [
    "Geometry", "rh_forward", "rh_adjoint", "rh_forward_entries", "rh_adjoint_entries",
    "build_oracle", "num_threads", "grad", "div", "tv_norm", "lap_symbol", "freq_norm",
    "precond_symbol", "precond_apply", "prox_dual", "tv_project", "conj_data_term",
    "make_descriptors", "power_beta", "power_c", "power_start", "PDRQState", "pdrq_solve", "cp_solve",
    "diagnostics", "pdrq_grad",
]
