"""GB300-native statistical model checking of mass-action reaction networks.

The hot path (Gillespie direct-method trajectories checked on the fly against a
time-bounded BLTLc formula, reduced into the Wilson score interval with the
iterative sample-size rule of Ballarini et al., PDMC 2009) runs in the CUDA
library ``_build/libsmc.so`` behind the C ABI of ``include/smc.h``.  This
package only marshals arguments to it; ``Context`` converts the seeded inputs
of ``workloads`` (networks, parameter sets, properties) into the ABI's arrays.
"""
from __future__ import annotations

import ctypes
import math
from typing import Dict, Optional, Sequence

import numpy as np

from . import _native as N
from ._native import (SMC_CONSERVATIVE, SMC_FIXED_N, SMC_ITERATIVE, SMC_MIXED,  # noqa: F401
                      SMC_PLAIN_FP64)


class SmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f'{N.smc_strerror(code).decode()} ({code}): {msg}')
        self.code = code


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy


def _stream(s):
    """cudaStream_t of a torch stream.  Torch's default stream has handle 0,
    which the C ABI reads as "the library's own stream"; pass the legacy
    default stream instead so the work is ordered with torch's."""
    return ctypes.c_void_p(s.cuda_stream or CUDA_STREAM_LEGACY)


def postfix(formula) -> list:
    """Formula tree of tuples (see ``workloads``) -> list of smc_node tuples."""
    out = []

    def rec(f):
        k = f[0]
        if k == 'atom':
            out.append((N.NODE['atom'], int(f[1]), 0.0, 0.0))
        elif k in ('true', 'false'):
            out.append((N.NODE[k], 0, 0.0, 0.0))
        elif k == 'not':
            rec(f[1]); out.append((N.NODE['not'], 0, 0.0, 0.0))
        elif k in ('and', 'or', 'implies'):
            rec(f[1]); rec(f[2]); out.append((N.NODE[k], 0, 0.0, 0.0))
        elif k == 'U':
            rec(f[3]); rec(f[4]); out.append((N.NODE['U'], 0, float(f[1]), float(f[2])))
        elif k in ('F', 'G', 'X'):
            rec(f[3]); out.append((N.NODE[k], 0, float(f[1]), float(f[2])))
        else:
            raise ValueError(f'unknown formula node {k!r}')

    rec(formula)
    return out


PRECISION = {'plain': SMC_PLAIN_FP64, 'fp64': SMC_PLAIN_FP64, 'mixed': SMC_MIXED}
SAMPLING = {'fixed': SMC_FIXED_N, 'iterative': SMC_ITERATIVE, 'conservative': SMC_CONSERVATIVE}


class Context:
    """One smc_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        N.load()
        h = ctypes.c_void_p()
        rc = N.smc_create(ctypes.byref(h), int(device))
        if rc != 0:
            raise SmcError(rc, 'smc_create')
        self.h = h
        self.device = device
        self.n_inst = 0
        self.s_max = 0

    def close(self):
        if getattr(self, 'h', None):
            N.smc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc, what):
        if rc != 0:
            raise SmcError(rc, f'{what}: {N.smc_last_error(self.h).decode()}')

    # -- loading --------------------------------------------------------------
    def load_model(self, model):
        reac = np.ascontiguousarray(model.reactants, np.int32)
        st = np.ascontiguousarray(model.stoich, np.int32)
        rates = np.ascontiguousarray(model.rates, np.float64)
        x0 = np.ascontiguousarray(model.x0, np.int32)
        self._check(N.smc_load_model(self.h, model.n_species, model.n_reactions, _p(reac, ctypes.c_int32),
                                     _p(st, ctypes.c_int32), _p(rates, ctypes.c_double),
                                     _p(x0, ctypes.c_int32), model.n_inst), 'smc_load_model')
        self.n_inst = model.n_inst
        self.s_max = model.n_species
        self._n_reactions = model.n_reactions
        self._feat = None  # smc_load_model resets the feature choice
        self._batch = None
        factors = list(getattr(model, 'factors', None) or [])
        if factors:
            self.load_rate_factors(factors)

    def load_rate_factors(self, factors):
        """Rate-law factors (reaction, species, power, a0, a1, b0, b1) for
        the loaded model (smc_load_rate_factors)."""
        fr = np.ascontiguousarray([f[0] for f in factors] or [0], np.int32)
        fs = np.ascontiguousarray([f[1] for f in factors] or [0], np.int32)
        fn = np.ascontiguousarray([f[2] for f in factors] or [1], np.int32)
        fp = np.ascontiguousarray([list(f[3:7]) for f in factors] or [[0.0, 0.0, 1.0, 0.0]], np.float64)
        self._check(N.smc_load_rate_factors(self.h, len(factors), _p(fr, ctypes.c_int32), _p(fs, ctypes.c_int32),
                                            _p(fn, ctypes.c_int32), _p(fp, ctypes.c_double)),
                    'smc_load_rate_factors')

    def load_batch(self, batch):
        ms = batch.models
        S = np.asarray([m.n_species for m in ms], np.int32)
        R = np.asarray([m.n_reactions for m in ms], np.int32)
        reac = np.ascontiguousarray(np.concatenate([m.reactants.ravel() for m in ms]), np.int32)
        st = np.ascontiguousarray(np.concatenate([m.stoich.ravel() for m in ms]), np.int32)
        rates = np.ascontiguousarray(np.concatenate([m.rates[0] for m in ms]), np.float64)
        x0 = np.ascontiguousarray(np.concatenate([m.x0[0] for m in ms]), np.int32)
        self._check(N.smc_load_model_batch(self.h, len(ms), _p(S, ctypes.c_int32), _p(R, ctypes.c_int32),
                                           _p(reac, ctypes.c_int32), _p(st, ctypes.c_int32),
                                           _p(rates, ctypes.c_double), _p(x0, ctypes.c_int32)),
                    'smc_load_model_batch')
        self.n_inst = len(ms)
        self.s_max = int(S.max())
        self._batch = batch

    def load_property(self, prop, t_max: float = math.inf, per_instance=None):
        """``prop``: a workloads.Property, or (after load_batch) a list of
        properties sharing one formula shape, one per instance."""
        if isinstance(prop, (list, tuple)):
            props = list(prop)
            formula = props[0].formula
            n_atoms = len(props[0].atoms)
            coef = np.ascontiguousarray(np.concatenate(
                [np.stack([a.coef for a in p.atoms]).ravel() for p in props]), np.int32)
            op = np.asarray([N.OP[a.op] for a in props[0].atoms], np.int32)
            bound = np.ascontiguousarray([a.bound for p in props for a in p.atoms], np.float64)
            per = 1
        else:
            formula = prop.formula
            n_atoms = len(prop.atoms)
            coef = np.ascontiguousarray(np.stack([a.coef for a in prop.atoms]) if n_atoms else
                                        np.zeros((1, 1)), np.int32)
            op = np.asarray([N.OP[a.op] for a in prop.atoms] or [0], np.int32)
            bound = np.asarray([a.bound for a in prop.atoms] or [0.0], np.float64)
            per = 0
            if self._batch is not None:
                coef = np.ascontiguousarray(np.concatenate([coef.ravel()] * self.n_inst), np.int32)
        nodes = postfix(formula)
        arr = (N.smc_node * len(nodes))(*[N.smc_node(*n) for n in nodes])
        self._check(N.smc_load_property(self.h, n_atoms, _p(coef, ctypes.c_int32), _p(op, ctypes.c_int32),
                                        _p(bound, ctypes.c_double), per, arr, len(nodes),
                                        float(t_max)), 'smc_load_property')
        atoms = props[0].atoms if isinstance(prop, (list, tuple)) else prop.atoms
        for a, at in enumerate(atoms):
            if at.lhs is not None:
                self.set_atom_expression(a, at.op, at.lhs, at.rhs)

    @staticmethod
    def _tokens(side):
        toks = []
        for t in side:
            k = N.TOK[t[0]]
            toks.append(N.smc_token(k, int(t[1]) if k in (0, 7) else 0, float(t[1]) if k == 1 else 0.0))
        return (N.smc_token * max(1, len(toks)))(*toks), len(toks)

    def set_atom_expression(self, atom: int, op: str, lhs, rhs):
        """Atom ``atom`` becomes the arithmetic atom lhs <op> rhs (token lists
        as in workloads.Atom; smc_set_atom_expression)."""
        la, ln = self._tokens(lhs)
        ra, rn = self._tokens(rhs)
        self._check(N.smc_set_atom_expression(self.h, int(atom), N.OP[op], la, ln, ra, rn),
                    'smc_set_atom_expression')

    def set_option(self, name: str, value: float):
        self._check(N.smc_set_option(self.h, N.OPT[name], float(value)), f'smc_set_option({name})')

    @property
    def monitor_kind(self) -> str:
        """'units' (the monitor automaton), 'trace' (the trace monitor, for
        formulas nested beyond the units) or 'none' (smc_monitor_kind)."""
        return {0: 'none', 1: 'units', 2: 'trace'}[N.smc_monitor_kind(self.h)]

    def cme_reach(self, instance: int = 0, cap: int = 1000, max_states: int = 2_000_000):
        """Exact P(property) by uniformisation (smc_cme_reach): dict p,
        truncated, poisson_tail, n_states, iterations, lambda_t."""
        r = N.smc_cme_result()
        self._check(N.smc_cme_reach(self.h, int(instance), int(cap), int(max_states), ctypes.byref(r)),
                    'smc_cme_reach')
        return r.as_dict()

    def launch_shapes(self, precision: str = 'mixed'):
        """The launches serving the loaded model (after an estimate or a
        simulation): list of dicts warps_per_block, blocks_per_sm, refill,
        n_instances, specialized."""
        out, i, n = [], 0, ctypes.c_int32(1)
        while i < n.value:
            w, b, r, m, sp = (ctypes.c_int32() for _ in range(5))
            self._check(N.smc_get_launch_shape(self.h, PRECISION[precision], i, ctypes.byref(n), ctypes.byref(w),
                                               ctypes.byref(b), ctypes.byref(r), ctypes.byref(m), ctypes.byref(sp)),
                        'smc_get_launch_shape')
            out.append(dict(warps_per_block=w.value, blocks_per_sm=b.value, refill=r.value, n_instances=m.value,
                            specialized=bool(sp.value)))
            i += 1
        return out

    # -- running --------------------------------------------------------------
    def estimate(self, confidence: float, half_width: float = 0.01, seed: int = 0,
                 precision: str = 'plain', sampling: str = 'iterative', fixed_n: int = 0):
        res = (N.smc_result * self.n_inst)()
        mode = PRECISION[precision] | SAMPLING[sampling]
        self._check(N.smc_estimate(self.h, float(confidence), float(half_width), int(seed), mode,
                                   int(fixed_n), res), 'smc_estimate')
        return [r.as_dict() for r in res]

    def get_verdicts(self, n: int) -> np.ndarray:
        out = np.zeros(n, np.uint8)
        self._check(N.smc_get_verdicts(self.h, _p(out, ctypes.c_uint8), n), 'smc_get_verdicts')
        return out

    def simulate(self, precision: str = 'plain', seed: int = 0, traj_begin: int = 0, n_traj: int = 1,
                 confidence: float = 0.95, outputs: Sequence[str] = ('verdict', 'status', 'events', 't_final'),
                 counts=None, wilson=None, stream=None) -> Dict[str, object]:
        """Runs trajectories [traj_begin, traj_begin + n_traj) of every
        instance on the GPU; returns torch CUDA tensors (counts [n_inst, 4],
        wilson [n_inst, 3] and the requested per-trajectory outputs)."""
        import torch
        dev = torch.device('cuda', self.device)
        n = self.n_inst
        out = {}
        if counts is None:
            counts = torch.zeros((n, 4), dtype=torch.int64, device=dev)
        out['counts'] = counts
        out['wilson'] = wilson if wilson is not None else torch.zeros((n, 3), dtype=torch.float64, device=dev)
        spec = dict(verdict=(torch.uint8, ()), status=(torch.uint8, ()), events=(torch.int64, ()),
                    t_final=(torch.float64, ()), x_final=(torch.int32, (self.s_max,)))
        so = N.smc_sim_out()
        so.counts = counts.data_ptr()
        so.wilson = out['wilson'].data_ptr()
        for k in outputs:
            dt, extra = spec[k]
            out[k] = torch.zeros((n, n_traj) + extra, dtype=dt, device=dev)
            setattr(so, k, out[k].data_ptr())
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        self._check(N.smc_simulate(self.h, PRECISION[precision], int(seed), int(traj_begin), int(n_traj),
                                   float(confidence), ctypes.byref(so), _stream(s)),
                    'smc_simulate')
        return out

    def simulate_snapshot(self, precision: str = 'mixed', seed: int = 0, traj_begin: int = 0, n_traj: int = 1,
                          t_snap: float = 5.0, stop: bool = False, stream=None) -> Dict[str, object]:
        """smc_simulate_snapshot: counts, verdict, status, snap, x_snap and
        e_snap (torch CUDA tensors, [n_inst, n_traj] / [n_inst, n_traj, S_max];
        e_snap holds int32 copies of the uint32 event counts)."""
        import torch
        dev = torch.device('cuda', self.device)
        n = self.n_inst
        out = dict(counts=torch.zeros((n, 4), dtype=torch.int64, device=dev),
                   verdict=torch.zeros((n, n_traj), dtype=torch.uint8, device=dev),
                   status=torch.zeros((n, n_traj), dtype=torch.uint8, device=dev),
                   snap=torch.zeros((n, n_traj), dtype=torch.uint8, device=dev),
                   x_snap=torch.zeros((n, n_traj, self.s_max), dtype=torch.int32, device=dev),
                   e_snap=torch.zeros((n, n_traj), dtype=torch.int32, device=dev))
        so = N.smc_sim_out()
        so.counts = out['counts'].data_ptr()
        so.verdict = out['verdict'].data_ptr()
        so.status = out['status'].data_ptr()
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        self._check(N.smc_simulate_snapshot(self.h, PRECISION[precision], int(seed), int(traj_begin), int(n_traj),
                                            float(t_snap), int(bool(stop)), ctypes.byref(so),
                                            ctypes.c_void_p(out['snap'].data_ptr()),
                                            ctypes.c_void_p(out['x_snap'].data_ptr()),
                                            ctypes.c_void_p(out['e_snap'].data_ptr()),
                                            _stream(s)), 'smc_simulate_snapshot')
        return out

    def set_features(self, species=None, with_rates: bool = True, log_rate_ref=None):
        """smc_set_features: which species (indices; None = all), whether the
        log-rate features follow, and their reference (None = the mean over
        the loaded instances)."""
        idx = np.ascontiguousarray([] if species is None else species, np.int32)
        ref = None if log_rate_ref is None else np.ascontiguousarray(log_rate_ref, np.float64)
        self._check(N.smc_set_features(self.h, idx.ctypes.data_as(ctypes.c_void_p) if idx.size else None,
                                       int(idx.size), int(bool(with_rates)),
                                       ref.ctypes.data_as(ctypes.c_void_p) if ref is not None else None),
                    'smc_set_features')
        self._feat = (idx.size or self.s_max) + 1 + (int(self._n_reactions) if with_rates else 0)

    def feature_count(self) -> int:
        return getattr(self, '_feat', None) or self.s_max + 1 + int(self._n_reactions)

    def snapshot_features(self, x_snap, t_snap: float, x_scale, t_scale: float, stream=None):
        """Features [n_inst * n_traj, F] (torch CUDA float32) of x_snap, F as
        set_features chose (default S + 1 + R)."""
        import torch
        n_traj = x_snap.shape[1]
        feat = torch.zeros((self.n_inst * n_traj, self.feature_count()), dtype=torch.float32,
                           device=x_snap.device)
        xs = np.ascontiguousarray(x_scale, np.float32)
        s = stream if stream is not None else torch.cuda.current_stream(x_snap.device)
        self._check(N.smc_snapshot_features(self.h, n_traj, ctypes.c_void_p(x_snap.data_ptr()), float(t_snap),
                                            xs.ctypes.data_as(ctypes.c_void_p), float(t_scale),
                                            ctypes.c_void_p(feat.data_ptr()), _stream(s)),
                    'smc_snapshot_features')
        return feat

    def estimate_cv(self, mlp, confidence: float, half_width: float, seed: int = 0, precision: str = 'mixed',
                    t_snap: float = 5.0, x_scale=None, t_scale: float = 30.0, beta: float = 1.0,
                    pilot: int = 2000):
        xs = np.ascontiguousarray(x_scale, np.float32)
        res = N.smc_cv_result()
        self._check(N.smc_estimate_cv(self.h, mlp.h, float(confidence), float(half_width), int(seed),
                                      PRECISION[precision], float(t_snap), xs.ctypes.data_as(ctypes.c_void_p),
                                      float(t_scale), float(beta), int(pilot), ctypes.byref(res)),
                    'smc_estimate_cv')
        return res.as_dict()

    def monitor_replay(self, paths, S: int):
        """paths: list of (x [n, S] ints, t [n] floats, tmin, closed)."""
        lens = np.asarray([len(p[1]) for p in paths], np.int32)
        x = np.ascontiguousarray(np.concatenate([np.asarray(p[0], np.int32).reshape(-1, S) for p in paths]),
                                 np.int32)
        t = np.ascontiguousarray(np.concatenate([np.asarray(p[1], np.float64) for p in paths]))
        tmin = np.asarray([p[2] for p in paths], np.float64)
        closed = np.asarray([1 if p[3] else 0 for p in paths], np.uint8)
        v = np.zeros(len(paths), np.int32)
        q = np.zeros(len(paths), np.int64)
        self._check(N.smc_monitor_replay(self.h, len(paths), _p(lens, ctypes.c_int32), _p(x, ctypes.c_int32),
                                         _p(t, ctypes.c_double), _p(tmin, ctypes.c_double),
                                         _p(closed, ctypes.c_uint8), _p(v, ctypes.c_int32),
                                         _p(q, ctypes.c_int64)), 'smc_monitor_replay')
        return v, q


class Mlp:
    """The surrogate network (smc_mlp_*): n_in -> 128 -> 128 -> 128 -> 1,
    BF16 tensor-core kernels, FP32 master weights, Adam."""
    NPARAM = N.SMC_MLP_NPARAM

    def __init__(self, n_in: int, device: int = 0, seed: int = 0):
        N.load()
        h = ctypes.c_void_p()
        rc = N.smc_mlp_create(ctypes.byref(h), int(device), int(n_in), int(seed))
        if rc != 0:
            raise SmcError(rc, 'smc_mlp_create')
        self.h = h
        self.n_in = n_in
        self.device = device

    def close(self):
        if getattr(self, 'h', None):
            N.smc_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != 0:
            raise SmcError(rc, f'{what}: {N.smc_mlp_last_error(self.h).decode()}')

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.NPARAM, np.float32)
        self._check(N.smc_mlp_get_params(self.h, out.ctypes.data_as(ctypes.c_void_p)), 'smc_mlp_get_params')
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == self.NPARAM
        self._check(N.smc_mlp_set_params(self.h, p.ctypes.data_as(ctypes.c_void_p)), 'smc_mlp_set_params')

    def gradient(self, x, y):
        """x: CUDA float32 [n, n_in], y: CUDA float32 [n] -> (grad [NPARAM], mean loss)."""
        import torch
        torch.cuda.current_stream(x.device).synchronize()  # the library runs this on its own stream
        g = np.zeros(self.NPARAM, np.float32)
        loss = np.zeros(1, np.float32)
        self._check(N.smc_mlp_gradient(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       int(x.shape[0]), g.ctypes.data_as(ctypes.c_void_p),
                                       loss.ctypes.data_as(ctypes.c_void_p)), 'smc_mlp_gradient')
        return g, float(loss[0])

    def train(self, x, y, epochs: int, batch: int = 4096, lr: float = 1e-3, seed: int = 0):
        import torch
        loss = np.zeros(epochs, np.float32)
        s = torch.cuda.current_stream(x.device)
        self._check(N.smc_mlp_train(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                    int(x.shape[0]), int(epochs), int(batch), float(lr), int(seed),
                                    loss.ctypes.data_as(ctypes.c_void_p), _stream(s)), 'smc_mlp_train')
        return loss

    def predict(self, x, skip=None, out=None):
        """smc_mlp_predict (or smc_mlp_predict_masked when skip, a uint8
        device tensor [n], is given: rows with skip != 0 keep out's values)."""
        import torch
        g = out if out is not None else torch.empty((x.shape[0],), dtype=torch.float32, device=x.device)
        s = torch.cuda.current_stream(x.device)
        if skip is None:
            self._check(N.smc_mlp_predict(self.h, ctypes.c_void_p(x.data_ptr()), int(x.shape[0]),
                                          ctypes.c_void_p(g.data_ptr()), _stream(s)),
                        'smc_mlp_predict')
        else:
            self._check(N.smc_mlp_predict_masked(self.h, ctypes.c_void_p(x.data_ptr()), int(x.shape[0]),
                                                 ctypes.c_void_p(skip.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                                 _stream(s)),
                        'smc_mlp_predict_masked')
        return g


def normal_quantile(p: float) -> float:
    return N.smc_normal_quantile(float(p))


def wilson_interval(yes: int, n: int, confidence: float):
    lo = ctypes.c_double()
    hi = ctypes.c_double()
    rc = N.smc_wilson_interval(int(yes), int(n), float(confidence), ctypes.byref(lo), ctypes.byref(hi))
    if rc != 0:
        raise SmcError(rc, 'smc_wilson_interval')
    return lo.value, hi.value


def wilson_sample(p: float, half_width: float, confidence: float) -> float:
    return N.smc_wilson_sample(float(p), float(half_width), float(confidence))
