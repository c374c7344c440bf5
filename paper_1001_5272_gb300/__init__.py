"""GB300-native in-place truncated Fourier transform (Harvey & Roche, 2010).

The compute path is the CUDA library built from ``csrc/`` (sm_103a), reached
through the C ABI of ``include/tft.h``; ``tft`` is its Python binding.
"""

from . import tft  # noqa: F401
from .tft import (Context, TFTError, tft_forward, tft_inverse,  # noqa: F401
                  tft_polymul, tft_forward_host, tft_inverse_host,
                  tft_polymul_host, tft_footprint, tft_describe_plan,
                  tft_last_error)
