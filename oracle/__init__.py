"""FP64 CPU oracle for the unbiased polyspectrum estimator.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the library.  See ``oracle.polyspectra``.
"""
from .polyspectra import *  # noqa: F401,F403
from .polyspectra import __all__  # noqa: F401
