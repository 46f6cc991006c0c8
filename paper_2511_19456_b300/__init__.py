"""B300-native engine for tree-level |M|^2 of multi-photon Compton scattering.

e-(p) gamma(k0) -> e-(p') + k gamma, evaluated at many phase-space points
through the node-reduced computable DAG of arXiv:2511.19456 on hand-written
sm_103a CUDA kernels behind a C-ABI (include/qed.h).

    from paper_2511_19456_b300 import Plan
    plan = Plan(k=4, summed=True, precision="fp64")
    m2 = plan.eval(momenta)          # momenta: cuda float64 [N, k+3, 4]
"""
from .api import (AbcPlan, Batch, Plan, TapePlan, reduction_steps, tape_export, cross_section, dag_counts, generate, measure_fma_peak,  # noqa: F401
                  schedule_export)
