"""GB300-native crack element method (CEM) step: C-ABI CUDA library + thin Python binding."""
from .binding import CEM, CEMError, load_library, probe_fp64_fma, probe_split, probe_split_rule, EXPORTED  # noqa: F401
from .build import build_library  # noqa: F401
