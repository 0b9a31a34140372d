"""FP64 CPU oracle for the sparse FCT (test infrastructure only; see fct_oracle)."""
from . import fct_oracle  # noqa: F401
