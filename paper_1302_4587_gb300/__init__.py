"""GB300-native local-max matching (Birn, Osipov, Sanders, Schulz, Sitchinava,
"Efficient Parallel and External Matching").

The compute path is liblm.so: hand-written sm_103a CUDA kernels behind the C
ABI of include/lm.h.  This package holds that library's sources (csrc/), its
in-tree build (_build.py) and a thin ctypes binding (binding.py) that takes
PyTorch tensors for device memory and streams.
"""
from .binding import (LM_DEVICE, LM_EAGAIN, LM_ECUDA, LM_EINVAL, LM_ENOMEM, LM_ENOTFOUND, LM_ETIMEOUT,
                      LM_F_ASYNC, LM_F_EDGE_CENTRIC, LM_F_PROFILE, LM_F_RENEW, LM_HOST, LM_K_COUNT, LM_K_INIT, LM_K_OTHER, LM_K_SWEEP, LM_K_CAND, LM_K_TAIL,
                      LM_K_VERTEX, LM_NIL, LM_NOALLOC_MAX_M, LM_NOALLOC_MAX_N, LM_OK, EXPORTS, BatchArgs, LmError, LmStats,
                      lm_batch_match, lm_create, lm_destroy, lm_graph_create, lm_graph_destroy, lm_graph_info,
                      lm_match, lm_match_small_noalloc, lm_poll, lm_strerror, lm_submit, lm_wait, load,
                      LmTuning, lm_autotune, lm_get_tuning, lm_set_tuning, lm_sync, lm_contract, lm_set_limits)
from ._build import build

__all__ = [n for n in dir() if n.startswith(("lm_", "LM_"))] + ["BatchArgs", "LmError", "LmStats", "LmTuning", "EXPORTS", "load", "build"]
