"""GB300 (sm_103a) data-driven S_n transport sweep (JSweep, arXiv 1803.09876).

The compute path is the CUDA library ``libjsweep.so`` behind the C ABI in
``include/jsweep.h``; ``jsweep`` is its thin Python binding.
"""

from . import jsweep  # noqa: F401
from .jsweep import (  # noqa: F401
    jsweep_build_dags,
    jsweep_mesh_create,
    jsweep_quadrature_create,
    jsweep_quadrature_product,
    jsweep_source_iterate,
    jsweep_sweep,
    mesh_from_dict,
)
