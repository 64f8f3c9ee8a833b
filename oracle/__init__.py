"""CPU FP64 oracle of the ensemble-of-4D-Var hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.
"""
from .eda_oracle import *  # noqa: F401,F403
