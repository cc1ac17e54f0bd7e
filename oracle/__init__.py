"""FP64 CPU oracle (test infrastructure; never used by the product path)."""
from . import rbf_oracle  # noqa: F401
