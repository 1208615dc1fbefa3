"""GB300 (sm_103a) state-vector library for the Mera method (arXiv 2411.15332).

The compute path is the CUDA library ``_build/libmera.so`` behind the C ABI
of ``include/mera.h``; this package is its Python binding.  Names are
resolved lazily so that ``paper_2411_15332_gb300.inputs`` (the seeded
workload generators) imports without touching the CUDA library.
"""

__all__ = ["State", "DAX", "DAS", "Batch", "AdjointExpectation", "gate_matrix", "launch_count", "profile_enable",
           "profile_read", "plan_summary", "rh_mvm", "RH_METHODS"]


def __getattr__(name):
    if name in ("State", "gate_matrix", "launch_count", "profile_enable", "profile_read", "plan_summary", "rh_mvm",
                "RH_METHODS"):
        from . import core
        return getattr(core, name)
    if name in ("Batch", "AdjointExpectation"):
        from . import qnn
        return getattr(qnn, name)
    if name in ("DAX", "DAS"):
        from . import compressed
        return getattr(compressed, name)
    raise AttributeError(name)
