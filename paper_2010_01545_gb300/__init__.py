"""GB300 (sm_103a) Piacsek-Williams momentum advection (MONC, Sec. 2.1).

``_abi`` mirrors the C ABI of ``include/advect.h`` function by function;
``torch_api`` wraps it for torch tensors and autograd.  The compute runs
only in the CUDA library ``_build/libadvect.so`` (built by ``build.build``);
a missing library is an error, never a fallback.
"""
from ._abi import (ADVECT_F16S, ADVECT_F32, ADVECT_F64, ADVECT_F64_FF, AdvectError, advect_adjoint,  # noqa: F401
                   advect_coeffs_from_grid, advect_create, advect_destroy,
                   advect_ensemble_adjoint, advect_ensemble_create, advect_ensemble_forward,
                   advect_f16s_output_scales, advect_forward, advect_forward_host,
                   advect_kernel_name, advect_last_error, advect_set_f64_levels, advect_sync,
                   advect_autotune, advect_tuned_config, advect_forward_noalloc,
                   library_path)


def __getattr__(name):
    if name in ("Advect", "AdvectFn", "AdvectEnsemble", "advect", "coefficients_from_grid"):
        from . import torch_api
        return getattr(torch_api, name)
    raise AttributeError(name)
