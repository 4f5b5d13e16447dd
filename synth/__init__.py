"""Seeded synthetic inputs shared by the oracle's tests, the CUDA path's tests and the bench.

This package builds parity-check matrices only (QC exponent matrices and PEG
graphs) and the job streams that use them.  It holds none of the decoding,
extraction or canonicalisation arithmetic: the oracle (``oracle/``) and the
CUDA library each implement those on their own from the inputs built here.
"""
from .codes import (  # noqa: F401
    Code,
    qc_code,
    csr_code,
    draw_qc,
    draw_qc_columns,
    peg,
    batch_codes,
    serving_codes,
    workload,
    WORKLOADS,
)
