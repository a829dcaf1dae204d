"""FP64 CPU oracle of the P3M gravity step -- test infrastructure only.

Imported only by tests/, __graft_entry__.smoke() and bench.py's CPU baseline and reference
arm.  The product path (paper_1510_07621_gb300) never imports, links or runs anything here.
"""
from .p3m_oracle import *  # noqa: F401,F403
from .p3m_oracle import Params  # noqa: F401
