"""Plain CPU oracle of RHSEG/HSEG -- test infrastructure only.

Used by tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py.
The library never imports this package.
"""
from .oracle import (MERGE_DTYPE, Level, OracleError, Result, build, compile_source, div_rn,  # noqa: F401
                     hseg_leaf, key, load, run)
