"""GB300 (sm_103a) solver library for variational phase-field fracture (AT1/AT2, P1 triangles).

The compute path is libpf.so (CUDA, C ABI in include/pf.h); this package only builds it and
marshals calls to it.  ``binding`` loads the library; ``sim`` wraps a resident simulation.
"""
__all__ = ["binding", "sim"]
