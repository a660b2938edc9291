"""GB300 (sm_103a) stochastic-LapH baryon blocks (arXiv:2211.16278).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/bblock.h``); :mod:`.bblock` is its Python binding.
"""
from .bblock import (BblockError, Context, CostModel, bblock_autotune,  # noqa: F401
                     bblock_compute, bblock_compute_batch, bblock_compute_host,
                     bblock_contract_noalloc, bblock_create, bblock_destroy,
                     bblock_from_triplet, bblock_get_option, bblock_last_error,
                     bblock_last_launch_count, bblock_last_path, bblock_last_wave_count,
                     bblock_mode_triplet, bblock_probe_fp64, bblock_profile_enable,
                     bblock_profile_read, bblock_set_option, bblock_status,
                     bblock_workspace_bytes, load)
