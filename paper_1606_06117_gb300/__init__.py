"""GB300 (sm_103a) multi-stage semi-Lagrangian advection: CIR, FEC, BEC and the
third-order CEC scheme of arXiv 1606.06117, as fused CUDA kernels behind the C
ABI of include/sl.h.

``paper_1606_06117_gb300.sl`` is the ctypes binding (argument marshalling
only); ``workloads`` draws the seeded synthetic inputs.  The binding is loaded
lazily so that the input generators import without a GPU.
"""
__all__ = ["sl", "workloads", "build"]


def __getattr__(name):
    if name == "sl":
        from . import _lib
        return _lib
    raise AttributeError(name)
