"""FP64 CPU oracle for the TACAW hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product path (the CUDA
library and its Python binding) never imports, links or executes it.
"""

from .tacaw_oracle import *  # noqa: F401,F403
