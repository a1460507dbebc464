"""GB300 (sm_103a) shadow-ray path of the Neural Intersection Function
(Fujieda, Kao & Harada, HPG 2023).

The CUDA library ``libnif.so`` (C ABI in ``include/nif.h``) does all the
work; ``paper_2306_07191_gb300.nif`` wraps it for PyTorch tensors and
``paper_2306_07191_gb300.synth`` draws the seeded synthetic inputs.  The
native library is loaded on first use of ``nif`` / ``_lib`` and importing
either fails loudly when it has not been built.
"""
__all__ = ["build", "synth", "workloads"]
