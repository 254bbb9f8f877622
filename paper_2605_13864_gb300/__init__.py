"""optigpu for GB300 (sm_103a): out-of-place matrix transpose and tree sum
reduction as hand-written CUDA kernels behind a C ABI (``include/optigpu.h``).

The two operations are the case studies of the thesis "Source-to-Source
Transformations for GPU Code Generation" (arxiv 2605.13864): the transpose
of Listing 3.5 (Sec. 3.1) and the sum of Listing 2.1 (Sec. 2.1).

Importing the package does not load the CUDA library; the first operation
does, and raises if the library cannot be built or loaded.
"""
from ._native import OptigpuError, load  # noqa: F401
from .api import (BatchPlan, Server, autotune, histogram, reduce_reserve, reduce_segmented, reduce_sum, scan, release_workspaces,  # noqa: F401
                  set_wait_limit_ns, stream_status, tma_eligible, transpose, transpose_batched, transpose_config_for, transpose_inplace, tune_configs,
                  tune_select, tune_selected)
