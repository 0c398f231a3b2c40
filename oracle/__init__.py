"""FP64 CPU oracle of the G-REST update -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this package.  The CUDA library never calls into it and the two
share no code.
"""
from .grest_oracle import *  # noqa: F401,F403
from .philox import gaussian_matrix, philox4x64_10  # noqa: F401
