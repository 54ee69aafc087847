"""GB300-native (sm_103a) MGARD+ hot path: multilevel decomposition and
recomposition of 1-4D tensor-product grids, level-wise quantization and the
labels' lossless stages (Liang et al., arXiv 2010.05872).

The compute lives in ``libmgardgb.so`` (CUDA, C ABI in include/mgard_gb.h);
``binding`` marshals arguments to it.  Importing the package does not load
the library; the first call does, and fails loudly when it is missing.
"""
from .binding import (  # noqa: F401
    F32, F64, MgardError, decompose, recompose, quantize, dequantize, value_range,
    workspace, mgard_num_levels, mgard_workspace_size, mgard_level_tolerances,
    decompose_4d, recompose_4d, quantize_4d, dequantize_4d,
    pack_labels, unpack_labels, huffman_encode, huffman_decode, label_entropy,
)
