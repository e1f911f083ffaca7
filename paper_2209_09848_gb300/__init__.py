"""GB300-native trajectory matched filter (Ganapathi 2022, Section 3.2).

The compute path is the CUDA library ``libmf.so`` (sources in ``csrc/``, ABI
in ``include/mf.h``); ``binding`` is a thin ctypes layer with the same names.
Nothing here falls back to a CPU implementation: if the library is missing
the binding raises.
"""
from .binding import (  # noqa: F401
    MFError, PrfTable, prf_table_create, prf_table_create_custom, search, search_workspace_size, search_noalloc,
    search_host, search_host_workspace_size, CANDIDATE_BYTES,
    rescore_topk, rescore_workspace_size, device_status, last_error, version, load, library_path,
    profile_enable, profile_read, decode_candidates, prf_plan, prf_bank, Batch,
    detect, detect_workspace_size, decode_detections, DETECTION_BYTES,
    background_refit, refit_workspace_size, wait_probe, wait_probe_search, search_status, MF_ETIMEOUT,
)
