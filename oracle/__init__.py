"""Oracle package -- test infrastructure only (see ``cuboid_oracle``).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it; the library never does.
"""
from .cuboid_oracle import *  # noqa: F401,F403
