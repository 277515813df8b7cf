"""GB300-native plane-wave H-psi / block-Davidson library (sm_103a CUDA behind a C ABI).

The compute path lives in libqm.so (see include/qm.h); this package is its thin Python
binding.  Importing it loads the library and raises if it is missing.
"""
from ._lib import load as _load

_load()

from .api import (Batch, GSpace, QMError, QM_FP64, QM_HPSI_NOALLOC_SCRATCH_BYTES, QM_MIXED, qm_gspace_create, qm_gspace_destroy,  # noqa: E402
                  QM_MLP_NPARAM, qm_batch_create, qm_davidson, qm_davidson_batched, qm_eigh_lowest, qm_zgemm, qm_mlp_forward, qm_mlp_loss_grad,
                  qm_mlp_pairs, qm_mlp_train, qm_precond_apply, qm_hpsi_prepare, qm_hamiltonian_diag, qm_gspace_indices, qm_gspace_query, qm_gspace_sticks, qm_hpsi, qm_hpsi_gamma, qm_hpsi_noalloc,
                  qm_tddft_etrs, qm_tddft_taylor, qm_gw_mel, qm_scf, qm_last_error,
                  qm_version)

__all__ = ["Batch", "qm_batch_create", "qm_davidson_batched", "QM_MLP_NPARAM", "qm_mlp_forward", "qm_mlp_loss_grad", "qm_mlp_pairs",
           "qm_mlp_train", "GSpace", "QMError", "QM_FP64", "QM_HPSI_NOALLOC_SCRATCH_BYTES", "QM_MIXED", "qm_gspace_create", "qm_gspace_destroy",
           "qm_davidson", "qm_eigh_lowest", "qm_zgemm", "qm_precond_apply", "qm_hpsi_prepare", "qm_hamiltonian_diag", "qm_gspace_indices", "qm_gspace_query", "qm_gspace_sticks", "qm_hpsi", "qm_hpsi_gamma", "qm_hpsi_noalloc", "qm_tddft_etrs", "qm_tddft_taylor", "qm_gw_mel", "qm_scf", "qm_last_error", "qm_version"]
