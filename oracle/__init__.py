"""FP64 CPU oracle for the SWiFT-IR block-matching step and its rendering step.

Test infrastructure only: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.
"""
from .swim import *  # noqa: F401,F403
from . import swim  # noqa: F401
from . import mir  # noqa: F401
from . import remod  # noqa: F401
from . import driver  # noqa: F401
