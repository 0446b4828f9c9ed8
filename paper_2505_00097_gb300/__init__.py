"""GB300-native FP64 BSSN hot path (arXiv 2505.00097): C-ABI library + thin binding."""
from . import workloads  # noqa: F401  (plain data; no compiled code)

__all__ = ["workloads", "binding", "build"]
