"""Plain FP64 CPU oracle for the level-dependent multigrid of Cools, Reps and
Vanroose, "A new level-dependent coarse grid correction scheme for indefinite
Helmholtz problems" (arXiv 1211.4752).

TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.  This package is the slow,
obviously correct restatement of the method that the CUDA library is checked
against.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  It shares no code, tables or helpers with
the CUDA path and imports nothing from it.

Every function is written in complex128 with numpy whole-array expressions that
follow the paper's definitions one step at a time (no fusion, blocking or
reordering beyond what the definition states).  ``helmholtz_mg`` holds the
method; each function cites the passage it follows.
"""

from .helmholtz_mg import *  # noqa: F401,F403
