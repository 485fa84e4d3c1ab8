"""GB300-native matrix-free Gauss-Newton step of PERF (Performant, Explicit
Radiance Fields): a C-ABI CUDA library (``libperf.so``, include/perf.h) and a
thin ctypes binding.  Importing the package loads the library; it raises if
the library has not been built (``python -m paper_2112_05598_gb300.build``)."""
from ._binding import (Batch, Context, LPC, Options, PerfError, block_jacobi, default_options,
                       load_library, measure_atomic_peak, upsample, PERF_F32, PERF_BF16, PERF_PRECOND_JACOBI,
                       PERF_PRECOND_BLOCK4, PERF_PRECOND_BLOCK_JACOBI, PERF_JUDGE_RESIDUAL,
                       PERF_JUDGE_OBJECTIVE)

__all__ = ["Batch", "Context", "LPC", "Options", "PerfError", "block_jacobi", "default_options",
           "load_library", "measure_atomic_peak", "upsample", "PERF_F32", "PERF_BF16", "PERF_PRECOND_JACOBI", "PERF_PRECOND_BLOCK4",
           "PERF_PRECOND_BLOCK_JACOBI", "PERF_JUDGE_RESIDUAL", "PERF_JUDGE_OBJECTIVE"]

load_library()
