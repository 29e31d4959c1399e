"""FP64 CPU oracle of the CGP quasigeostrophic time step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library never does, and it shares
no code with the CUDA path.  See ``qg_oracle.py`` for the functions and the
passages of the paper each one follows.

Parity status of each function is stated in its test file; the long-run
statistics of the chaotic flow (time-mean energy over tens of time units) are
"parity unpinned": the paper prints no number for them.
"""
from .qg_oracle import *  # noqa: F401,F403
from . import qg_oracle  # noqa: F401
