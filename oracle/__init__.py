"""FP64 CPU oracle (test infrastructure; see nk_oracle's header)."""
from .nk_oracle import *  # noqa: F401,F403
