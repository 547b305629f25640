"""GB300-native range-SVD (Zoom-SVD, arXiv 1805.00754): C-ABI CUDA library + binding."""
from .zoomsvd import Store, Server, QueryOut, ZsError, load_library, launch_count  # noqa: F401
