"""GB300 (sm_103a) recycled Krylov solves of shifted systems (A + gamma_l E_k) x = b.

The compute path is the C-ABI library librecyc.so (hand-written CUDA); this
package holds its sources (csrc/), its build script and a thin ctypes binding.
"""
from . import recyc  # noqa: F401
from .recyc import (RS_FP64, RS_INIT, RS_MIXED, RS_UPDATE, Problem, RecycError, load,  # noqa: F401
                    make_desc, rs_synthesize_data, rs_workspace_bytes)
