"""CPU oracle for the statistical model checking hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.  It
shares no code with the CUDA path (it reads the same seeded inputs from
``workloads``, nothing else).

``smc_oracle.c`` holds the arithmetic (Philox4x32-10, the SSA direct method of
Sec. 2.2, the BLTLc semantics of Sec. 3.1 evaluated on the stored trace, the
normal quantile); ``wilson.py`` holds Eq. 4, Eq. 5 and the iterative procedure
of Fig. 2.  This module only marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, 'smc_oracle.c')
_BUILD = os.path.join(_HERE, '_build')
_LIB = os.path.join(_BUILD, 'liborc.so')
_lock = threading.Lock()
_lib = None

KINDS = {'true': 0, 'false': 1, 'atom': 2, 'not': 3, 'and': 4, 'or': 5, 'implies': 6,
         'U': 7, 'F': 8, 'G': 9, 'X': 10}
OPS = {'<': 0, '<=': 1, '>=': 2, '>': 3, '==': 4, '!=': 5}
V_F, V_T, V_U = 0, 1, 2


class _Node(ctypes.Structure):
    _fields_ = [('kind', ctypes.c_int32), ('c0', ctypes.c_int32), ('c1', ctypes.c_int32),
                ('arg', ctypes.c_int32), ('lo', ctypes.c_double), ('hi', ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile smc_oracle.c with gcc (-O2 -ffp-contract=off) into _build/."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f'.{os.getpid()}.tmp'
        subprocess.check_call(['gcc', '-O2', '-ffp-contract=off', '-fPIC', '-shared', '-pthread',
                               '-o', tmp, _SRC, '-lm'])
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER
        L.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32)] * 3
        L.orc_u01.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        L.orc_u01.restype = ctypes.c_double
        L.orc_normal_quantile.argtypes = [ctypes.c_double]
        L.orc_normal_quantile.restype = ctypes.c_double
        L.orc_eval_prefix.restype = ctypes.c_int
        L.orc_run.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for counter (4 words) and key (2 words)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                            _ptr(o, ctypes.c_uint32))
    return o


def u01(hi: int, lo: int) -> float:
    return lib().orc_u01(hi, lo)


def normal_quantile(p: float) -> float:
    return lib().orc_normal_quantile(p)


def flatten_formula(formula):
    """Tree of tuples -> (node array, root index)."""
    nodes = []

    def rec(f):
        k = f[0]
        c0 = c1 = arg = -1
        lo = hi = 0.0
        if k == 'atom':
            arg = int(f[1])
        elif k in ('not',):
            c0 = rec(f[1])
        elif k in ('and', 'or', 'implies'):
            c0 = rec(f[1]); c1 = rec(f[2])
        elif k == 'U':
            lo, hi = float(f[1]), float(f[2])
            c0 = rec(f[3]); c1 = rec(f[4])
        elif k in ('F', 'G', 'X'):
            lo, hi = float(f[1]), float(f[2])
            c0 = rec(f[3])
        elif k not in ('true', 'false'):
            raise ValueError(f'unknown formula node {k!r}')
        nodes.append((KINDS[k], c0, c1, arg, lo, hi))
        return len(nodes) - 1

    root = rec(formula)
    arr = (_Node * len(nodes))(*[_Node(*n) for n in nodes])
    return arr, root


class _Token(ctypes.Structure):
    _fields_ = [('kind', ctypes.c_int32), ('arg', ctypes.c_int32), ('value', ctypes.c_double)]


TOKEN_KIND = {'x': 0, 'c': 1, '+': 2, '-': 3, '*': 4, '/': 5, 'sqrt': 6, 'pow': 7}


def _expr_arrays(prop):
    """Arithmetic atoms as (expr_ptr [n+1], n_lhs [n], tokens) or Nones."""
    if not any(a.lhs is not None for a in prop.atoms):
        return None, None, None
    ptr, nl, toks = [0], [], []
    for a in prop.atoms:
        if a.lhs is None:
            nl.append(0)
        else:
            nl.append(len(a.lhs))
            for t in list(a.lhs) + list(a.rhs):
                k = TOKEN_KIND[t[0]]
                toks.append((k, int(t[1]) if k in (0, 7) else 0, float(t[1]) if k == 1 else 0.0))
        ptr.append(len(toks))
    arr = (_Token * max(1, len(toks)))(*[_Token(*t) for t in toks])
    return np.asarray(ptr, np.int32), np.asarray(nl, np.int32), arr


def _atom_arrays(prop, S):
    n = len(prop.atoms)
    coef = np.zeros((max(n, 1), S), np.int32)
    op = np.zeros(max(n, 1), np.int32)
    bound = np.zeros(max(n, 1), np.float64)
    for i, a in enumerate(prop.atoms):
        coef[i, :] = a.coef
        op[i] = OPS[a.op]
        bound[i] = a.bound
    return n, coef, op, bound


def eval_prefix(prop, S: int, x: np.ndarray, t: np.ndarray, tmin: float, closed: bool,
                tmin_exact: bool = False) -> int:
    """Kleene value (0 false, 1 true, 2 undetermined) of ``prop`` at position 0
    of a prefix with states x[n,S] and entry times t[n]; later positions have
    entry time >= tmin (the next one exactly tmin when ``tmin_exact``), or do
    not exist when ``closed``."""
    x = np.ascontiguousarray(x, np.int32).reshape(-1, S)
    t = np.ascontiguousarray(t, np.float64)
    nodes, root = flatten_formula(prop.formula)
    n_at, coef, op, bound = _atom_arrays(prop, S)

    eptr, enl, etok = _expr_arrays(prop)

    class F(ctypes.Structure):
        _fields_ = [('n_nodes', ctypes.c_int), ('root', ctypes.c_int),
                    ('nodes', ctypes.POINTER(_Node)), ('n_atoms', ctypes.c_int), ('S', ctypes.c_int),
                    ('coef', ctypes.POINTER(ctypes.c_int32)), ('op', ctypes.POINTER(ctypes.c_int32)),
                    ('bound', ctypes.POINTER(ctypes.c_double)), ('expr_ptr', ctypes.POINTER(ctypes.c_int32)),
                    ('n_lhs', ctypes.POINTER(ctypes.c_int32)), ('tokens', ctypes.POINTER(_Token))]

    f = F(len(nodes), root, nodes, n_at, S, _ptr(coef, ctypes.c_int32), _ptr(op, ctypes.c_int32),
          _ptr(bound, ctypes.c_double), _ptr(eptr, ctypes.c_int32) if eptr is not None else None,
          _ptr(enl, ctypes.c_int32) if enl is not None else None, etok)
    L = lib()
    L.orc_eval_prefix.argtypes = [ctypes.POINTER(F), ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_int32), ctypes.c_double, ctypes.c_int, ctypes.c_int]
    return L.orc_eval_prefix(ctypes.byref(f), t.shape[0], _ptr(t, ctypes.c_double),
                             _ptr(x, ctypes.c_int32), float(tmin), int(bool(closed)), int(bool(tmin_exact)))


def _factor_arrays(model):
    """Rate-law factors of a workloads.Model as (reaction, species, power,
    params[n][4]) arrays (empty for pure mass action)."""
    fac = list(getattr(model, 'factors', None) or [])
    fr = np.ascontiguousarray([f[0] for f in fac] or [0], np.int32)
    fs = np.ascontiguousarray([f[1] for f in fac] or [0], np.int32)
    fn = np.ascontiguousarray([f[2] for f in fac] or [1], np.int32)
    fp = np.ascontiguousarray([f[3:7] for f in fac] or [[0.0, 0.0, 1.0, 0.0]], np.float64)
    if not fac:
        fr, fs, fn, fp = fr[:0], fs[:0], fn[:0], fp[:0]
    return fr, fs, fn, fp


def run(model, prop, seed: int, instance: int = 0, traj_begin: int = 0, n_traj: int = 1,
        budget: int = 1 << 40, t_max: float = float('inf'), threads: Optional[int] = None,
        want_x: bool = False):
    """Simulate and verify trajectories traj_begin .. traj_begin+n_traj-1 of
    one instance of ``model`` (a workloads.Model; instance ``instance`` picks
    its rate and x0 row, and keys the random numbers).

    Returns a dict of numpy arrays: verdict (uint8), status (uint8: 0 decided,
    1 budget, 2 error), events (uint64), t_final (float64) and, if
    ``want_x``, x_final (int32 [n, S])."""
    S, R = model.n_species, model.n_reactions
    row = instance if model.n_inst > 1 else 0
    rates = np.ascontiguousarray(model.rates[row], np.float64)
    x0 = np.ascontiguousarray(model.x0[row], np.int32)
    reac = np.ascontiguousarray(model.reactants, np.int32)
    st = np.ascontiguousarray(model.stoich, np.int32)
    nodes, root = flatten_formula(prop.formula)
    n_at, coef, op, bound = _atom_arrays(prop, S)
    eptr, enl, etok = _expr_arrays(prop)
    fr, fs, fn, fp = _factor_arrays(model)
    n = int(n_traj)
    out = dict(verdict=np.zeros(n, np.uint8), status=np.zeros(n, np.uint8),
               events=np.zeros(n, np.uint64), t_final=np.zeros(n, np.float64))
    if want_x:
        out['x_final'] = np.zeros((n, S), np.int32)
    if threads is None:
        threads = os.cpu_count() or 1
    L = lib()
    P = ctypes.POINTER
    L.orc_run.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32),
                          P(ctypes.c_double), P(ctypes.c_int32), ctypes.c_int, P(ctypes.c_int32),
                          P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                          P(_Node), ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32),
                          P(ctypes.c_double), P(ctypes.c_int32), P(ctypes.c_int32), P(_Token), ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                          ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                          P(ctypes.c_uint8), P(ctypes.c_uint8), P(ctypes.c_uint64),
                          P(ctypes.c_double), P(ctypes.c_int32)]
    rc = L.orc_run(S, R, _ptr(reac, ctypes.c_int32), _ptr(st, ctypes.c_int32),
                   _ptr(rates, ctypes.c_double), _ptr(x0, ctypes.c_int32), len(fr),
                   _ptr(fr, ctypes.c_int32), _ptr(fs, ctypes.c_int32), _ptr(fn, ctypes.c_int32),
                   _ptr(fp, ctypes.c_double), len(nodes), root, nodes,
                   n_at, _ptr(coef, ctypes.c_int32), _ptr(op, ctypes.c_int32),
                   _ptr(bound, ctypes.c_double), _ptr(eptr, ctypes.c_int32) if eptr is not None else None,
                   _ptr(enl, ctypes.c_int32) if enl is not None else None, etok,
                   int(seed) & ((1 << 64) - 1), int(instance),
                   int(traj_begin), n, int(budget), float(t_max), int(threads),
                   _ptr(out['verdict'], ctypes.c_uint8), _ptr(out['status'], ctypes.c_uint8),
                   _ptr(out['events'], ctypes.c_uint64), _ptr(out['t_final'], ctypes.c_double),
                   _ptr(out['x_final'], ctypes.c_int32) if want_x else None)
    if rc != 0:
        raise RuntimeError('oracle: a trajectory failed (allocation or undecided path)')
    return out
