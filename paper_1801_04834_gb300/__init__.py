"""GB300-native FX correlator hot path (Cobalt, arXiv 1801.04834): polyphase
filter bank, fine delay + bandpass correction, X-stage correlation.

The compute runs in libfx_gb300.so (hand-written CUDA for sm_103a) behind the
C ABI of include/fx.h; this package only marshals arguments (`_abi`) and
offers a torch-tensor convenience layer (`Correlator`). PyTorch supplies
device memory and streams."""
from ._abi import (FX_BF16, FX_CI8, FX_CI16, FX_F16, FX_F16_SPLIT, FX_F32, FX_TF32_SPLIT, FxError,  # noqa: F401
                   load, last_error)
from .api import Correlator, f32_block, f32_unblock  # noqa: F401
