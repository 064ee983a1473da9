"""GB300 (sm_103a) preconditioned DCA for the graph Ginzburg-Landau model.

The solver lives in the CUDA library ``_build/libpdca.so`` (sources in
``csrc/``, interface in ``include/pdca.h``); ``binding`` is its thin ctypes
binding and ``build`` compiles it.
"""

from . import binding  # noqa: F401
from .binding import Problem, make_params, params_from_workload, PdcaError  # noqa: F401
