"""GB300-native (sm_103a) SIMP stiffness assembly and compliance sensitivities.

Per iteration of density-based topology optimisation (SOPTX, arXiv 2505.02438,
Sec. 2.2) the library assembles K(rho) = sum_e E(rho_e) K_e^0 into a fixed CSR
pattern and computes dc_e = -E'(rho_e) u_e^T K_e^0 u_e on one GPU, behind the C
ABI in include/soptx.h.  Import is light: the CUDA library loads on first use.
"""
from . import workloads  # noqa: F401


def __getattr__(name):
    if name in ("Mesh", "version", "host_plan", "step_group"):
        from . import api
        return getattr(api, name)
    if name == "Compliance":
        from . import autograd
        return autograd.Compliance
    raise AttributeError(name)
