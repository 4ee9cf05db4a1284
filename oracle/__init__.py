"""CPU FP64 oracle (test infrastructure only; see fe_oracle's header)."""
from . import fe_oracle  # noqa: F401
