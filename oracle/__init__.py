"""FP64 CPU oracle of the exact-exchange operator (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The CUDA product path never does.
"""

from .exx_oracle import *  # noqa: F401,F403
from .exx_oracle import __all__  # noqa: F401
