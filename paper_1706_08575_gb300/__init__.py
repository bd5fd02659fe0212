"""GB300-native frame theoretic convolutional gridding (weighted 2-D adjoint NUFFT).

The compute lives in libftcg.so (C ABI, include/ftcg.h, CUDA kernels for sm_103a); this package
only builds it and marshals arguments to it.
"""
from .ftcg import (BF16X2, C64, F32, F64, LAYOUT_AUTO, LAYOUT_DUPLICATE,  # noqa: F401
                   LAYOUT_HALO, MLP_PARAMS, PREC_BF16, PREC_FP32, SPREAD_AUTO, SPREAD_BLOCK,
                   SPREAD_TENSOR, SPREAD_WINDOW, WINDOW_ES, WINDOW_GAUSS, WINDOW_KB, Batch,
                   FtcgError, Mlp, Plan, features, features_batch, lib, lib_path)
