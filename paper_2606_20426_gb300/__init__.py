"""GB300 (sm_103a) implementation of the TaCauchy hot path: one implicit
incremental-potential-contact step of a tetrahedral gel pad pressed by a rigid
indenter, then Cauchy-stress extraction, traction, pressure and the pixel map
(TaCauchy, Sec. III-B/III-C, Algorithms 1-2).

The compute lives in libtacauchy.so (CUDA, C ABI in include/tacauchy.h);
``tacauchy`` is its ctypes binding.  Build with
``python -m paper_2606_20426_gb300.build``.
"""
from . import tacauchy  # noqa: F401
from .tacauchy import (Env, Server, TcError, autotune_pcg, load, pcg_shape, step_batch,  # noqa: F401
                       stress_from_F, extract_batch)
