"""Oracle package -- test infrastructure only (see ``cuboid_oracle``).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of ``bench.py``
may import it; the library never does.  ``oracle.paper_loop`` (imported on its own) is
the C/OpenMP restatement of the paper's section 5 loop, the timed CPU baseline.
"""
from .cuboid_oracle import *  # noqa: F401,F403
