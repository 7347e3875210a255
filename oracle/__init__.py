"""FP64 CPU oracle (test infrastructure only; see copa_oracle.py)."""
from .copa_oracle import *  # noqa: F401,F403
from .copa_oracle import slices_to_tensor  # noqa: F401
