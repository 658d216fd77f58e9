"""FP64 CPU oracle (test infrastructure only; see eot_oracle.py)."""
from . import eot_oracle  # noqa: F401
