"""GB300 (sm_103a) solver for ACA H-matrix RWG/EFIE systems with the symmetric near-field
Schur-complement preconditioner of arXiv 2111.13483.  The arithmetic lives in
libhmsolve.so (csrc/); ``hmsolve`` is its ctypes binding."""
from . import hmsolve
from .hmsolve import (hmat_create, precond_setup, solve, solve_device, hmat_stats, hm_last_error, hmat_destroy,
                      hm_get_order, hm_get_fill, hm_get_block, hm_apply, hm_get_index_map, hm_profile,
                      hm_get_profile, hm_plan_order, hm_plan_fill, hm_test_hold, Batch, HMError)
