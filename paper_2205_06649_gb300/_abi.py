"""ctypes declarations of the C ABI in include/dd4dvar.h (argument marshalling only).

The shared library is built in-tree (paper_2205_06649_gb300/libdd4dvar.so, see
build.py).  There is no fallback: if the library is missing or fails to load,
importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdd4dvar.so")

c_double_p = C.POINTER(C.c_double)
c_int_p = C.POINTER(C.c_int)
c_ll_p = C.POINTER(C.c_longlong)


class dd4dv_model(C.Structure):
    _fields_ = [("nlon", C.c_int), ("nlat", C.c_int),
                ("lat_min_deg", C.c_double), ("lat_max_deg", C.c_double),
                ("radius", C.c_double), ("gravity", C.c_double), ("omega", C.c_double),
                ("dt", C.c_double), ("nsteps", C.c_int), ("precision", C.c_int),
                ("h_ref", C.c_double)]


class dd4dv_decomp(C.Structure):
    _fields_ = [("P1", C.c_int), ("P2", C.c_int), ("Q", C.c_int),
                ("lon_cuts", c_int_p), ("lat_cuts", c_int_p), ("t_cuts", c_int_p),
                ("o_lon", C.c_int), ("o_lat", C.c_int), ("o_t", C.c_int),
                ("mu", C.c_double), ("lambda_", C.c_double), ("weight_obs", C.c_int),
                ("cluster", C.c_int), ("ckpt_k", C.c_int)]


class dd4dv_solver(C.Structure):
    _fields_ = [("lbfgs_m", C.c_int), ("max_local_iters", C.c_int), ("max_trials", C.c_int),
                ("max_outer", C.c_int), ("eps_outer", C.c_double), ("gtol_rel", C.c_double),
                ("c1", C.c_double), ("use_graphs", C.c_int), ("local_solver", C.c_int),
                ("gn_iters", C.c_int), ("cg_iters", C.c_int), ("cg_tol", C.c_double)]


class dd4dv_stats(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("evals", C.c_longlong), ("sub_evals", C.c_longlong),
                ("pt_steps", C.c_longlong), ("dw_inf", C.c_double), ("J_sum", C.c_double),
                ("gnorm_rel_max", C.c_double), ("n_linesearch_fail", C.c_int)]


STATUS = {0: "DD4DV_OK", -1: "DD4DV_EINVAL", -2: "DD4DV_ENOMEM", -3: "DD4DV_ECUDA",
          -4: "DD4DV_ESTATE", -5: "DD4DV_ETIMEOUT", -6: "DD4DV_ENONFINITE", 1: "DD4DV_NOTCONV"}

_CTX = C.c_void_p
_P = C.c_void_p     # any data pointer (host or device)

PROTOTYPES = {
    "dd4dv_create": (C.c_int, [C.POINTER(dd4dv_model), C.c_void_p, C.POINTER(_CTX)]),
    "dd4dv_destroy": (C.c_int, [_CTX]),
    "dd4dv_set_background": (C.c_int, [_CTX, _P]),
    "dd4dv_set_background_error": (C.c_int, [_CTX, _P, C.c_double, C.c_int]),
    "dd4dv_set_observations": (C.c_int, [_CTX, C.c_longlong, _P, _P, _P, _P, _P, _P]),
    "dd4dv_set_decomposition": (C.c_int, [_CTX, C.POINTER(dd4dv_decomp)]),
    "dd4dv_num_subdomains": (C.c_int, [_CTX, c_int_p]),
    "dd4dv_control_layout": (C.c_int, [_CTX, _P, _P]),
    "dd4dv_eval": (C.c_int, [_CTX, _P, _P, _P, _P, C.c_int]),
    "dd4dv_eval_forward": (C.c_int, [_CTX, _P, _P, _P, C.c_int]),
    "dd4dv_eval_backward": (C.c_int, [_CTX, _P, _P, C.c_int]),
    "dd4dv_tlm": (C.c_int, [_CTX, _P, _P, _P, C.c_int]),
    "dd4dv_adjoint": (C.c_int, [_CTX, _P, _P, _P, C.c_int]),
    "dd4dv_gn_hessvec": (C.c_int, [_CTX, _P, _P, _P, C.c_int]),
    "dd4dv_traj_layout": (C.c_int, [_CTX, _P]),
    "dd4dv_trajectories": (C.c_int, [_CTX, _P, _P, C.c_int]),
    "dd4dv_exchange": (C.c_int, [_CTX, _P, C.c_int]),
    "dd4dv_reset_exchange": (C.c_int, [_CTX]),
    "dd4dv_boundary_trajectory": (C.c_int, [_CTX, _P, C.c_int]),
    "dd4dv_forward": (C.c_int, [_CTX, _P, _P, C.c_int]),
    "dd4dv_observe": (C.c_int, [_CTX, _P, C.c_longlong, _P, _P, _P, _P, _P, C.c_int]),
    "dd4dv_outer_step": (C.c_int, [_CTX, C.POINTER(dd4dv_solver), C.POINTER(dd4dv_stats)]),
    "dd4dv_run": (C.c_int, [_CTX, C.POINTER(dd4dv_solver), _P, C.POINTER(dd4dv_stats)]),
    "dd4dv_analysis": (C.c_int, [_CTX, _P, C.c_int]),
    "dd4dv_get_controls": (C.c_int, [_CTX, _P, C.c_int]),
    "dd4dv_set_controls": (C.c_int, [_CTX, _P, C.c_int]),
    "dd4dv_pt_steps": (C.c_int, [_CTX, c_ll_p]),
    "dd4dv_launch_count": (C.c_int, [_CTX, c_ll_p]),
    "dd4dv_cluster_size": (C.c_int, [_CTX, c_int_p]),
    "dd4dv_sweep_config": (C.c_int, [_CTX, _P, c_double_p]),
    "dd4dv_profile_sweeps": (C.c_int, [_CTX, _P, C.c_int, _P]),
    "dd4dv_set_sweep_config": (C.c_int, [_CTX, _P]),
    "dd4dv_set_sweep_variant": (C.c_int, [_CTX, C.c_int, C.c_int]),
    "dd4dv_set_owned": (C.c_int, [_CTX, _P]),
    "dd4dv_tz_forward": (C.c_int, [_CTX, C.c_int, C.c_int, C.c_double, _P, _P, C.c_int]),
    "dd4dv_tz_tlm": (C.c_int, [_CTX, C.c_int, C.c_int, C.c_double, _P, _P, _P, C.c_int]),
    "dd4dv_tz_adjoint": (C.c_int, [_CTX, C.c_int, C.c_int, C.c_double, _P, _P, _P, C.c_int]),
    "dd4dv_tz_eval": (C.c_int, [_CTX, C.c_int, C.c_int, C.c_double, _P, _P, _P, C.c_int]),
    "dd4dv_checkpoint_interval": (C.c_int, [_CTX, c_int_p, c_double_p]),
    "dd4dv_stage1_stored": (C.c_int, [_CTX, c_int_p, c_double_p]),
    "dd4dv_local_solve": (C.c_int, [_CTX, C.POINTER(dd4dv_solver), C.POINTER(dd4dv_stats)]),
    "dd4dv_sweep_kernels": (C.c_int, [_CTX, _P]),
    "dd4dv_forward_noalloc": (C.c_int, [C.POINTER(dd4dv_model), _P, _P, C.c_void_p]),
    "dd4dv_last_error": (C.c_char_p, [_CTX]),
}


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib
