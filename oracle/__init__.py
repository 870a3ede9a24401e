"""FP64 CPU oracle (test infrastructure only; see pf_oracle)."""
from .pf_oracle import *  # noqa: F401,F403
