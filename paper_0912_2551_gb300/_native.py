"""ctypes binding of the C ABI in include/smc.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  The shared
library is built in-tree by ``paper_0912_2551_gb300/build.py``; if it is
missing, loading raises (there is no fallback implementation).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, '_build', 'libsmc.so')

SMC_OK = 0
SMC_E_INVALID_ARG = -1
SMC_E_OOM = -2
SMC_E_CUDA = -3
SMC_E_UNSUPPORTED = -4
SMC_E_STATE = -5
SMC_E_NO_DEVICE = -6
SMC_STATUS_BUDGET = 1
SMC_PLAIN_FP64 = 0
SMC_MIXED = 1
SMC_FIXED_N = 0 << 4
SMC_ITERATIVE = 1 << 4
SMC_CONSERVATIVE = 2 << 4
NODE = dict(true=0, false=1, atom=2, **{'not': 3, 'and': 4, 'or': 5, 'implies': 6}, U=7, F=8, G=9, X=10)
OP = {'<': 0, '<=': 1, '>=': 2, '>': 3, '==': 4, '!=': 5}
OPT = dict(event_budget=0, renorm_log2=1, autotune=2, warps_per_block=3, blocks_per_sm=4, selection=8,
           refill=5, record=6, jit=7, trace_cap=9)

c_i32p = ctypes.POINTER(ctypes.c_int32)
c_u8p = ctypes.POINTER(ctypes.c_uint8)
c_f64p = ctypes.POINTER(ctypes.c_double)
c_i64p = ctypes.POINTER(ctypes.c_int64)


class smc_node(ctypes.Structure):
    _fields_ = [('kind', ctypes.c_int32), ('arg', ctypes.c_int32), ('lo', ctypes.c_double),
                ('hi', ctypes.c_double)]


class smc_result(ctypes.Structure):
    _fields_ = [('p_hat', ctypes.c_double), ('lo', ctypes.c_double), ('hi', ctypes.c_double),
                ('n', ctypes.c_uint64), ('yes', ctypes.c_uint64), ('launched', ctypes.c_uint64),
                ('events', ctypes.c_uint64), ('budget_hits', ctypes.c_uint64),
                ('status', ctypes.c_int32), ('iterations', ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class smc_sim_out(ctypes.Structure):
    _fields_ = [('counts', ctypes.c_void_p), ('wilson', ctypes.c_void_p), ('verdict', ctypes.c_void_p),
                ('status', ctypes.c_void_p), ('events', ctypes.c_void_p), ('t_final', ctypes.c_void_p),
                ('x_final', ctypes.c_void_p)]


class smc_cv_result(ctypes.Structure):
    _fields_ = [('p_hat', ctypes.c_double), ('lo', ctypes.c_double), ('hi', ctypes.c_double),
                ('n_eff', ctypes.c_double), ('var', ctypes.c_double), ('beta', ctypes.c_double),
                ('n_full', ctypes.c_uint64), ('n_prefix', ctypes.c_uint64), ('events_full', ctypes.c_uint64),
                ('events_prefix', ctypes.c_uint64),
                ('iterations', ctypes.c_int32), ('status', ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class smc_token(ctypes.Structure):
    _fields_ = [('kind', ctypes.c_int32), ('arg', ctypes.c_int32), ('value', ctypes.c_double)]


TOK = {'x': 0, 'c': 1, '+': 2, '-': 3, '*': 4, '/': 5, 'sqrt': 6, 'pow': 7}


class smc_cme_result(ctypes.Structure):
    _fields_ = [('p', ctypes.c_double), ('truncated', ctypes.c_double), ('poisson_tail', ctypes.c_double),
                ('n_states', ctypes.c_int64), ('iterations', ctypes.c_int64), ('lambda_t', ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


SMC_MLP_NPARAM = 35329
SMC_MLP_MAX_BATCH = 4194304
c_f32p = ctypes.POINTER(ctypes.c_float)

_lib = None

# name -> (restype, argtypes)
SIGNATURES = {
    'smc_create': (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]),
    'smc_destroy': (None, [ctypes.c_void_p]),
    'smc_strerror': (ctypes.c_char_p, [ctypes.c_int]),
    'smc_last_error': (ctypes.c_char_p, [ctypes.c_void_p]),
    'smc_load_model': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, c_i32p, c_i32p,
                                      c_f64p, c_i32p, ctypes.c_int]),
    'smc_load_model_batch': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_i32p, c_i32p, c_i32p,
                                            c_i32p, c_f64p, c_i32p]),
    'smc_load_property': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_i32p, c_i32p, c_f64p,
                                         ctypes.c_int, ctypes.POINTER(smc_node), ctypes.c_int,
                                         ctypes.c_double]),
    'smc_set_option': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]),
    'smc_monitor_kind': (ctypes.c_int, [ctypes.c_void_p]),
    'smc_cme_reach': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int64,
                                     ctypes.POINTER(smc_cme_result)]),
    'smc_set_atom_expression': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(smc_token), ctypes.c_int,
                                               ctypes.POINTER(smc_token), ctypes.c_int]),
    'smc_load_rate_factors': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_i32p, c_i32p, c_i32p, c_f64p]),
    'smc_get_launch_shape': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, c_i32p, c_i32p, c_i32p,
                                            c_i32p, c_i32p, c_i32p]),
    'smc_estimate': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                    ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(smc_result)]),
    'smc_get_verdicts': (ctypes.c_int, [ctypes.c_void_p, c_u8p, ctypes.c_uint64]),
    'smc_simulate': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(smc_sim_out),
                                    ctypes.c_void_p]),
    'smc_simulate_noalloc': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(smc_sim_out),
                                            ctypes.c_void_p]),
    'smc_monitor_replay': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_i32p, c_i32p, c_f64p, c_f64p,
                                          c_u8p, c_i32p, c_i64p]),
    'smc_simulate_snapshot': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                             ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                                             ctypes.POINTER(smc_sim_out), ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p]),
    'smc_set_features': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p]),
    'smc_snapshot_features': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_double,
                                             ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    'smc_mlp_create': (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_uint64]),
    'smc_mlp_destroy': (None, [ctypes.c_void_p]),
    'smc_mlp_last_error': (ctypes.c_char_p, [ctypes.c_void_p]),
    'smc_mlp_get_params': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    'smc_mlp_set_params': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    'smc_mlp_gradient': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    'smc_mlp_train': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_uint64, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    'smc_mlp_predict': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    'smc_mlp_predict_masked': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p]),
    'smc_estimate_cv': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                       ctypes.c_float, ctypes.c_double, ctypes.c_uint64,
                                       ctypes.POINTER(smc_cv_result)]),
    'smc_log_fp64': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    'smc_div_fp64': (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    'smc_normal_quantile': (ctypes.c_double, [ctypes.c_double]),
    'smc_wilson_interval': (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, c_f64p,
                                           c_f64p]),
    'smc_wilson_sample': (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    'smc_fig2_next_batch': (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.POINTER(ctypes.c_uint64)]),
}


def load(build_if_missing: bool = True):
    """Loads libsmc.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing:
            from . import build as _build
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f'CUDA library not built: {LIB_PATH}')
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _mk(name):
    def call(*args):
        return getattr(load(), name)(*args)
    call.__name__ = name
    call.__doc__ = f'Calls {name} of include/smc.h.'
    return call


for _n in SIGNATURES:
    globals()[_n] = _mk(_n)
