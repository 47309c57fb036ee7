"""GB300 (sm_103a) shift-free 2D FMM for the log potential (arXiv 2009.00767).

``paper_2009_00767_gb300.binding`` is the ctypes binding of include/fmm.h;
``paper_2009_00767_gb300.build`` compiles libfmm.so; ``inputs`` draws seeded
synthetic particle systems.
"""
__all__ = ["binding", "build", "inputs"]
