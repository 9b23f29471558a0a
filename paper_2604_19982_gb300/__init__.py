"""GB300-native (sm_103a) polyhedral spatial join: the refinement hot path of
3DPipe (arXiv 2604.19982) behind a C ABI (``include/pj.h``).

``paper_2604_19982_gb300.pj`` is the ctypes binding; ``build.py`` compiles
the CUDA library in-tree.
"""
from . import build  # noqa: F401


def load():
    """Import the binding (raises if ``libpj.so`` has not been built)."""
    from . import pj
    pj.lib()
    return pj
