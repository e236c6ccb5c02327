"""GB300-native Householder Dice (arXiv 2101.07464): matrix-free y = M_t x for Ginibre and
Haar random matrices, as hand-written CUDA kernels for sm_103a behind the C ABI of
include/hd.h.  `binding` is the thin Python layer over libhd.so; `build` compiles it."""
from .binding import (HD, HDBatch, hd_first_product_noalloc, hd_create_batched, hd_get_batch_layout, HD_F32, HD_F64, HD_GINIBRE, HD_HAAR, HDError, hd_apply, hd_create,
                      hd_destroy, hd_get_counts, hd_get_device_bytes, hd_philox_normals,
                      hd_philox_words, hd_probe, hd_reset, hd_run, hd_sync, hd_set_options, lib, library_path,
                      make_run_spec, hd_profile_enable, hd_profile_read,
                      hd_get_launches)

__all__ = ["HD", "HDBatch", "hd_first_product_noalloc", "hd_create_batched", "hd_get_batch_layout", "HDError", "hd_create", "hd_set_options", "hd_apply", "hd_probe", "hd_reset", "hd_run", "hd_sync", "make_run_spec", "hd_profile_enable", "hd_profile_read", "hd_get_launches",
           "hd_destroy", "hd_get_counts", "hd_get_device_bytes", "hd_philox_normals",
           "hd_philox_words", "lib", "library_path", "HD_GINIBRE", "HD_HAAR", "HD_F64", "HD_F32"]
