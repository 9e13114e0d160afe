"""FP64 CPU oracle (test infrastructure only; see ids_oracle)."""
from .ids_oracle import *  # noqa: F401,F403
