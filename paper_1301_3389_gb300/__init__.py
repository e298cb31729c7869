"""GB300 (sm_103a) library for the Diagonalized Newton Algorithm (DNA) for KL-NMF.

The compute path is libdna.so (hand-written CUDA, C ABI in include/dna.h); this package
is its thin Python binding.  Importing it fails if the library has not been built.
"""
from ._lib import (  # noqa: F401
    DNA_BF16, DNA_ENGINE_AUTO, DNA_ENGINE_SIMT, DNA_ENGINE_TENSOR, DNA_ERR_ALLOC, DNA_ERR_ARG,
    DNA_ERR_CUDA, DNA_ERR_LIMIT, DNA_ERR_NONFINITE, DNA_KL_NOALLOC_MAX_PARTIALS, DNA_ERR_TIMEOUT, DNA_ERR_UNSUPPORTED, DNA_F32, DNA_F64,
    DNA_OK, LIB, LIB_PATH, DNAError, dna_bind, dna_bind_csr, dna_create, dna_create_sparse, dna_default_opts, dna_destroy,
    dna_get_choice, dna_get_costs, dna_get_status, dna_iterate, dna_kl, dna_kl_backward, dna_kl_noalloc, dna_step_H_fixed, dna_step_H_adjoint, dna_step_H_adjoint_w, dna_normalize,
    dna_opts, dna_phase_times, dna_profile, dna_profile_phases, dna_run_host, PHASES, dna_set_stream, dna_step_H, dna_step_W, dna_strerror, make_opts,
    mu_step, mu_iterate, dna_group_create, dna_group_bind, dna_group_set_stream,
    dna_group_normalize, dna_group_step_H, dna_group_step_W, dna_group_iterate,
    dna_group_use_graph, dna_group_autotune, dna_group_tile_config, dna_group_kl, dna_group_get_status, dna_group_get_choice,
    dna_group_launches_per_iteration, dna_group_destroy, dna_shard_rowsums,
    dna_shard_set_rowsums, dna_shard_H_begin, dna_shard_H_end, dna_shard_W_begin,
    dna_shard_W_pass1, dna_shard_W_pass2, dna_shard_W_end, DNA_SELECT_PAPER, DNA_SELECT_DESCENT,
    dna_set_selection, dna_use_graph)
