"""CPU oracle for BP + LSD (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product path (``paper_2406_18655_gb300``) never
does.  See ``oracle/oracle.cpp`` for what each function restates and where in
the paper it comes from.
"""
from .oracle import *  # noqa: F401,F403
