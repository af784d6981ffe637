"""FP64 CPU oracle (test infrastructure only; see revo_oracle)."""
from .revo_oracle import *  # noqa: F401,F403
from . import revo_oracle  # noqa: F401
