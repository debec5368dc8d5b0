"""GB300-native two-phase general-pressure-equation solver (Huang, arXiv 2011.00814).

The compute path is the CUDA library ``libgpe2p.so`` behind the C ABI declared
in ``include/gpe2p.h``; :mod:`paper_2011_00814_gb300.gpe2p` is its ctypes
binding and :mod:`paper_2011_00814_gb300.inputs` builds seeded workloads.
Submodules are imported lazily so that the input generators can be used
without loading the CUDA library.
"""
__all__ = ["gpe2p", "inputs"]
