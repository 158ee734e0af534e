"""GB300 (sm_103a) solver for l1-regularised conditional Gaussian graphical models by
alternating Newton coordinate descent (McCarter & Kim, AISTATS 2016, Algorithm 1).

The compute path is the CUDA library ``libcggm.so`` (C ABI in include/cggm.h); this
package is its Python binding.  Build it with ``paper_1509_04681_gb300.build.build()``.
"""
from .cggm import (  # noqa: F401
    Server,
    footprint,
    Context,
    CGGMError,
    cggm_opts,
    cggm_info,
    make_opts,
    opts_default,
    LIB_PATH,
    EXPORTED,
    CGGM_FP64,
    CGGM_F32,
    CGGM_F64,
    CGGM_BF16,
    CGGM_I8_GENO,
    CGGM_SWEEP_BATCH_AUTO,
    tuned_batch,
    tuner_save,
    tuner_load,
    partition_columns,
    partition_theta_columns,
    chol_symbolic,
    chol_supernodes,
    chol_structure,
    block_order,
    permute_csr,
    CGGM_ORDER_NATURAL,
    CGGM_ORDER_RCM,
    CGGM_ORDER_GIVEN,
    CGGM_ORDER_MINDEG,
    CGGM_MIXED,
    CGGM_OK,
    CGGM_EMAXITER,
    CGGM_ENOTPD,
    CGGM_EINVAL,
    CGGM_ELINESEARCH,
)
