"""FP64 CPU oracle for the trajectory matched filter (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library.  See ``oracle/oracle.py`` (the search), ``oracle/detect.py`` (score
normalisation and candidates) and ``oracle/background.py`` (the per-pixel
background re-fit) for the functions and their citations.
"""
from .oracle import *  # noqa: F401,F403
from .detect import *  # noqa: F401,F403
from .background import *  # noqa: F401,F403
