"""FP64 CPU oracle (test infrastructure; see ba_oracle's header)."""
from .ba_oracle import *  # noqa: F401,F403
