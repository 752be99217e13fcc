"""CPU FP64 oracle for the BLDTT compute phase.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the library.  See bldtt_oracle.py for
the passages of the paper each function follows and the readings taken, and
learned.py for the learned pair selector and the multi-degree BLDTT.
"""
from .bldtt_oracle import *  # noqa: F401,F403
from .bldtt_oracle import (COULOMB, YUKAWA, OSCILLATORY, REG_COULOMB, TEST_POLY, PP, PC,  # noqa: F401
                           CP, CC, FULL, CC_PP_ONLY, Result, SampledBLDTT, Tree)
