"""FP64 CPU oracle (test infrastructure only; see fde_oracle's header)."""
from .fde_oracle import *  # noqa: F401,F403
