"""FP64 CPU oracle for the visibility path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
Python binding) never imports, links or runs anything here, and shares no code
with it.  See ``oracle.c`` for what is computed and the conventions used.
"""
from .oracle import (OracleProblem, build, oracle_vis, oracle_enu, oracle_strength,
                     oracle_voltage, rel_l2)

__all__ = ["OracleProblem", "build", "oracle_vis", "oracle_enu", "oracle_strength",
           "oracle_voltage", "rel_l2"]
