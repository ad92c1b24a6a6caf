"""FP64 CPU oracle (test infrastructure only; see hom_oracle)."""
from . import hom_oracle  # noqa: F401
