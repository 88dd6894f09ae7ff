"""GB300-native data-parallel partially coherent ptychographic engine (arXiv 2406.06640).

The compute path is libptycho.so (hand-written CUDA for sm_103a) behind the C
ABI of include/ptycho.h; `binding` marshals arguments with ctypes and
`engine.Reconstruction` accepts torch CUDA tensors.
"""
from .binding import (  # noqa: F401
    BLUR_AMPLITUDE,
    ENGINE_DM,
    ENGINE_PIE,
    BLUR_INTENSITY,
    EXPORTED,
    FARFIELD,
    NEARFIELD,
    GenSpec,
    Plan,
    PtychoError,
    PtychoParams,
    UNet,
    generate,
    library_path,
    load,
    make_gen_spec,
    make_params,
    permutation,
    set_batch_chunk,
    set_staged_chunk,
    version,
)

__version__ = "0.1.0"
