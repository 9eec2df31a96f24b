"""FP64 CPU oracle for the GeoSSTV P-PDS hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg and reference arm, never by the
``paper_2510_00562_gb300`` package.  See ``oracle/ppds.py``.
"""
from .ppds import *  # noqa: F401,F403
from .ppds import Params, State  # noqa: F401
