"""GB300-native fast direct solver for high-order FEM Dirichlet Poisson problems.

After Zlotnik & Zlotnik, arXiv:1609.07758 (algorithm (a) of Sect. 2 par. 4 with the
fast F_n-transforms of Theorem 2).  The compute path is the C-ABI library
``lib/libhofem.so`` (hand-written CUDA for sm_103a, declared in ``include/hofem.h``);
this package only loads it and marshals arguments (see ``binding``).  There is no CPU
fallback: calls fail with ``HofemError`` when the library cannot be loaded.
"""
from .binding import (  # noqa: F401
    HOFEM_BF16,
    HOFEM_BF16_REFINED,
    HOFEM_FP16,
    HOFEM_FP16_REFINED,
    HOFEM_FP32,
    HOFEM_FP32_REFINED,
    HOFEM_FP64,
    HOFEM_SWEEP_FORWARD,
    HOFEM_SWEEP_FUSED,
    HOFEM_SWEEP_INVERSE,
    Batch,
    HofemError,
    Plan,
    batch_partition,
    hofem_apply,
    hofem_apply_static,
    hofem_autotune,
    hofem_copy_block,
    hofem_destroy,
    hofem_get_eigen,
    hofem_get_info,
    hofem_get_profile,
    hofem_profile,
    hofem_last_error,
    hofem_plan,
    hofem_reserve,
    hofem_residual,
    hofem_set_refinement,
    hofem_solve,
    hofem_status_string,
    hofem_sweep,
    hofem_transform1d,
    library_path,
    load_library,
)
