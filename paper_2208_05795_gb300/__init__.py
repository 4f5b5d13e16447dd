"""GB300-native trapping-set enumeration for QC-LDPC codes.

The hot path of the modified Cole importance-sampling method (arXiv
2208.05795, Sec. III) as a CUDA library for sm_103a with a C ABI
(include/tsx.h); this package is its thin Python binding.
"""
from ._tsx import (  # noqa: F401
    DECODERS,
    Batch,
    Code,
    Server,
    TsList,
    TsxError,
    batch_create,
    batch_free,
    batch_run,
    batch_stats,
    batch_view,
    code_info,
    cycle_counts,
    decode_thresholds_noalloc,
    emd_spectrum,
    enum_params_default,
    enumerate_ts,
    free_code,
    free_ts_list,
    is_fer_estimate,
    is_params_default,
    lib,
    lnms_decode,
    lnms_params,
    lnms_simulate,
    load_code,
    make_params,
    measure_peaks,
    server_params_default,
    strerror,
    ts_list_stats,
    ts_list_view,
    tune_tile,
    union_bound_fer,
)
