"""GB300 (sm_103a) pseudospectral Taylor-Couette time step (nsCouette method).

The compute path is libtc.so (CUDA kernels behind the C ABI of include/tc.h);
``paper_1908_00587_gb300.tc`` is its ctypes binding.  Build with
``python -c "import __graft_entry__ as g; g.build()"`` from the repository root.
"""
from .build import LIB as LIB_PATH  # noqa: F401


def load():
    """Import and return the binding module (raises if libtc.so is missing)."""
    from . import tc
    return tc
