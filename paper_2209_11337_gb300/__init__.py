"""QMC conditional-pathwise Greeks on NVIDIA GB300 (sm_103a).

The product is ``libqmccpw.so`` (CUDA kernels behind the C-ABI in
``include/qmccpw.h``); ``paper_2209_11337_gb300.qmccpw`` is its Python
binding and ``paper_2209_11337_gb300.build`` compiles it.
"""
from . import qmccpw  # noqa: F401
from .qmccpw import QmcCpwError  # noqa: F401
