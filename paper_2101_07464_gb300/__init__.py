"""GB300-native Householder Dice (arXiv 2101.07464): matrix-free y = M_t x for Ginibre and
Haar random matrices, as hand-written CUDA kernels for sm_103a behind the C ABI of
include/hd.h.  `binding` is the thin Python layer over libhd.so; `build` compiles it;
`autograd` differentiates whole trajectories through the library's reverse mode."""
from .binding import (HD, HDBatch, HDComplex, HDError, USV, HD_F32, HD_F64, HD_GINIBRE, HD_HAAR, hd_adjoint_enable,
                      hd_adjoint_position, hd_adjoint_restart, hd_adjoint_step, hd_apply, hd_autotune, hd_check_bounded_wait,
                      hd_create,
                      hd_create_batched, hd_destroy, hd_first_product_noalloc, hd_fp64_fma_rate, hd_get_batch_layout,
                      hd_get_counts, hd_get_device_bytes, hd_get_launches, hd_get_map_options,
                      hd_get_tuning, hd_goe_apply, hd_philox_normals,
                      hd_philox_words, hd_probe, hd_probe_at, hd_profile_enable, hd_profile_read, hd_reset, hd_run,
                      hd_set_engine, hd_set_options, hd_set_trial_sigmas, hd_set_tuning, hd_sync, hd_usv_apply, lib, library_path,
                      make_run_spec)

__all__ = ["HD", "HDBatch", "HDComplex", "HDError", "USV", "HD_F32", "HD_F64", "HD_GINIBRE", "HD_HAAR",
           "hd_adjoint_enable", "hd_adjoint_position", "hd_adjoint_restart", "hd_adjoint_step",
           "hd_apply", "hd_autotune", "hd_check_bounded_wait", "hd_create", "hd_create_batched", "hd_destroy", "hd_first_product_noalloc", "hd_fp64_fma_rate",
           "hd_get_batch_layout", "hd_get_counts", "hd_get_device_bytes", "hd_get_launches",
           "hd_get_map_options", "hd_get_tuning", "hd_goe_apply", "hd_philox_normals", "hd_philox_words", "hd_probe", "hd_probe_at", "hd_profile_enable",
           "hd_profile_read", "hd_reset", "hd_run", "hd_set_engine", "hd_set_options", "hd_set_trial_sigmas", "hd_set_tuning",
           "hd_sync", "hd_usv_apply", "lib",
           "library_path", "make_run_spec"]
