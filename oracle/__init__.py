"""CPU float64 oracle for entropic optimal transport and SK-NR.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The library (``paper_2506_14780_gb300``) never calls
it: there is no CPU fallback.  The oracle shares no code with the CUDA path;
the only module both read is ``workloads`` (seeded random inputs).

The oracle is a plain, slow, obviously-correct restatement of the paper in
NumPy float64: each function names the equation, algorithm or section it
follows.  Parity status of each function is listed in ``eot_oracle``'s header.
"""
from .eot_oracle import *  # noqa: F401,F403
from .eot_oracle import __all__  # noqa: F401
