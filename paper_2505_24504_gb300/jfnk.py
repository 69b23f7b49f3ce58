"""ctypes binding of include/jfnk.h.  Argument marshalling only: every step of
the path runs in libjfnk.so.  Device arrays are torch CUDA tensors (float64,
contiguous); the stream is torch's current stream unless one is given."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def lib_path() -> str:
    return os.path.join(HERE, "libjfnk.so")


class JfnkError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib().jfnk_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("nz", C.c_int), ("x0", C.c_double), ("x1", C.c_double),
                ("z0", C.c_double), ("z1", C.c_double), ("periodic_x", C.c_int)]


class Physics(C.Structure):
    _fields_ = [("cp", C.c_double), ("cv", C.c_double), ("g", C.c_double), ("p0", C.c_double),
                ("theta0", C.c_double), ("mu", C.c_double), ("background", C.c_int),
                ("ubg", C.c_double), ("wbg", C.c_double), ("N_bv", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("newton_tol", C.c_double), ("newton_max", C.c_int), ("gmres_restart", C.c_int),
                ("gmres_max", C.c_int), ("ew_gamma", C.c_double), ("ew_alpha", C.c_double),
                ("ew_eta0", C.c_double), ("ew_eta_max", C.c_double), ("mg_key", C.c_char * 16),
                ("fv_levels", C.c_int), ("massfix", C.c_int), ("transfer_l2", C.c_int), ("precond_prec", C.c_int),
                ("sigma_fv", C.c_double), ("sigma_dg", C.c_double), ("c_ip", C.c_double),
                ("use_graphs", C.c_int), ("tile_faces", C.c_int), ("tile_volume", C.c_int),
                ("tile_fv", C.c_int), ("fv_split_cells", C.c_int), ("profile", C.c_int),
                ("precond_fd_eps", C.c_double), ("time_budget_ms", C.c_double), ("dg_fused", C.c_int),
                ("rk_stages", C.c_int), ("rk_alpha", C.c_double * 4)]

    @classmethod
    def defaults(cls, **kw):
        o = cls()
        _lib().jfnk_default_opts(C.byref(o))
        for k, v in kw.items():
            if k == "mg_key":
                v = v.encode() if isinstance(v, str) else v
            if k == "rk_alpha":
                v = (C.c_double * 4)(*(list(v) + [0.0] * (4 - len(v))))
            setattr(o, k, v)
        return o


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("stages", C.c_int), ("newton_its", C.c_int), ("gmres_its", C.c_int),
                ("dg_calls", C.c_int), ("fv_calls", C.c_int), ("res0", C.c_double), ("res_final", C.c_double),
                ("t_precond_ms", C.c_double), ("t_jv_ms", C.c_double), ("t_orth_ms", C.c_double),
                ("t_newton_ms", C.c_double), ("reorth", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def _lib():
    global _LIB
    if _LIB is None:
        p = lib_path()
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is not built; run __graft_entry__.build() (nvcc, sm_103a)")
        L = C.CDLL(p)
        P, D, I, S = C.c_void_p, C.c_double, C.c_int, C.c_size_t
        sig = {
            "jfnk_default_opts": (None, [P]),
            "jfnk_create": (I, [P, I, P, P, C.POINTER(C.c_void_p)]),
            "jfnk_destroy": (None, [P]),
            "jfnk_num_unknowns": (S, [P]),
            "jfnk_workspace_bytes": (S, [P, I, P]),
            "jfnk_node_coords": (I, [P, P, P]),
            "jfnk_init_state": (I, [P, P, P, P]),
            "dg_residual": (I, [P, P, P, P]),
            "jv_product": (I, [P, P, P, P, D, D, P, P]),
            "mg_precondition": (I, [P, P, D, P, P, P]),
            "implicit_step": (I, [P, P, D, I, P, P]),
            "jfnk_fv_levels": (I, [P]),
            "jfnk_fv_level_size": (I, [P, I, C.POINTER(I), C.POINTER(I)]),
            "jfnk_transfer_to_fv": (I, [P, P, P, P]),
            "jfnk_transfer_to_dg": (I, [P, P, P, P]),
            "jfnk_fv_residual": (I, [P, I, P, P, P]),
            "jfnk_eos_pressure": (I, [P, P, S, P, P]),
            "jfnk_norm2": (I, [P, P, S, P, P]),
            "jfnk_batch_create": (I, [P, I, I, C.POINTER(C.c_void_p)]),
            "jfnk_batch_destroy": (None, [P]),
            "jfnk_batch_step": (I, [P, P, P, P, P, P]),
            "jfnk_batch_dg_residual": (I, [P, P, P, P]),
            "jfnk_batch_set_mode": (I, [P, I]),
            "jfnk_batch_last_launches": (I, [P, P, P, P, P]),
            "jfnk_batch_last_times": (I, [P, P]),
            "jfnk_norm2_noalloc": (I, [P, S, P, P]),
            "jfnk_time_operator": (I, [P, I, P, P, I, P, P]),
            "jfnk_tangent_product": (I, [P, P, P, D, P, P]),
            "jfnk_launch_count": (C.c_ulonglong, []),
            "jfnk_autotune": (I, [P, P, P, I, P, P, P]),
            "jfnk_strerror": (C.c_char_p, [I]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


lib = _lib


BATCH_STREAMS, BATCH_LOCKSTEP, BATCH_LOCKSTEP_UNGROUPED = 0, 1, 2


class Batch:
    """Ensemble members stepped together (jfnk_batch_*): concurrently on their own
    streams (mode BATCH_STREAMS) or in lock-step with one grouped launch per
    operator across members (BATCH_LOCKSTEP)."""

    def __init__(self, contexts, max_threads=0, mode=BATCH_STREAMS):
        self.contexts = list(contexts)
        arr = (C.c_void_p * len(self.contexts))(*[c.h.value for c in self.contexts])
        h = C.c_void_p()
        _check(_lib().jfnk_batch_create(arr, len(self.contexts), int(max_threads), C.byref(h)),
               "jfnk_batch_create")
        self.h = h
        if mode != BATCH_STREAMS:
            self.set_mode(mode)

    def set_mode(self, mode):
        _check(_lib().jfnk_batch_set_mode(self.h, int(mode)), "jfnk_batch_set_mode")

    def last_launches(self):
        """{launches, grouped, member_launches, rounds} of the last lock-step step."""
        v = [C.c_ulonglong() for _ in range(4)]
        _check(_lib().jfnk_batch_last_launches(self.h, *[C.byref(x) for x in v]), "jfnk_batch_last_launches")
        d = dict(zip(("launches", "grouped", "member_launches", "rounds"), [x.value for x in v]))
        t = (C.c_double * 3)()
        _check(_lib().jfnk_batch_last_times(self.h, t), "jfnk_batch_last_times")
        d.update(ms_members=t[0], ms_issue=t[1], ms_device=t[2])
        return d

    def close(self):
        if getattr(self, "h", None):
            _lib().jfnk_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _member_states(self, *lists):
        """Per (arrays, name): one contiguous float64 CUDA state per member, of that
        member's size (every count, dtype and length checked before the rest)."""
        for states, what in lists:
            if len(states) != len(self.contexts):
                raise ValueError(f"{what}: {len(states)} arrays for {len(self.contexts)} members")
            for c, t in zip(self.contexts, states):
                _vec(t, c.N, what)
        for states, _ in lists:
            for t in states:
                _ptr(t)

    def jfnk_batch_step(self, states, dts, schemes, raise_on_error=True):
        n = len(self.contexts)
        self._member_states((states, "states"))
        if len(dts) != n or len(schemes) != n:
            raise ValueError(f"dts and schemes need one entry per member ({n})")
        U = (C.c_void_p * n)(*[s.data_ptr() for s in states])
        dt = (C.c_double * n)(*[float(x) for x in dts])
        sc = (C.c_int * n)(*[int(x) for x in schemes])
        status = (C.c_int * n)()
        stats = (Stats * n)()
        rc = _lib().jfnk_batch_step(self.h, U, dt, sc, status, stats)
        if raise_on_error:
            _check(rc, "jfnk_batch_step")
        return list(status), list(stats)

    def jfnk_batch_dg_residual(self, states, outs, stream=None):
        """f_m = M^-1 L_h(U_m) for all members: one face and one volume launch per
        (order, viscous) group of members."""
        n = len(self.contexts)
        self._member_states((states, "states"), (outs, "outs"))
        U = (C.c_void_p * n)(*[_ptr(s).value for s in states])
        f = (C.c_void_p * n)(*[_ptr(o).value for o in outs])
        _check(_lib().jfnk_batch_dg_residual(self.h, U, f, _stream(stream)), "jfnk_batch_dg_residual")


def _check_norm_args(x, out, n):
    """float64 vectors and 0 <= n <= x.numel(), checked before anything is launched
    (a wrong dtype or length would make the kernel read past the buffer)."""
    import torch
    n = x.numel() if n is None else int(n)
    if x.dtype != torch.float64 or out.dtype != torch.float64:
        raise ValueError("x and out must be float64")
    if n < 0 or n > x.numel() or out.numel() < 1:
        raise ValueError(f"n = {n} outside [0, {x.numel()}] or empty out")
    return n


def norm2_noalloc(x, out, n=None, stream=None):
    """|x|_2 into out[0] without a context or any device allocation (fixed
    in-library scratch; see include/jfnk.h)."""
    n = _check_norm_args(x, out, n)
    _check(_lib().jfnk_norm2_noalloc(_ptr(x), n, _ptr(out), _stream(stream)), "jfnk_norm2_noalloc")


def launch_count() -> int:
    return int(_lib().jfnk_launch_count())


def _vec(t, n, what, at_least=False):
    """t unchanged after checking that it is float64 with n elements (at least n
    with at_least).  The library indexes every array by the context's sizes, so a
    shorter or narrower tensor would be read or written past its end: refuse it
    before anything is launched.  None passes (optional arguments)."""
    import torch
    if t is None:
        return t
    if t.dtype != torch.float64:
        raise ValueError(f"{what}: expected float64, got {t.dtype}")
    if t.numel() < n or (not at_least and t.numel() != n):
        raise ValueError(f"{what}: expected {'at least ' if at_least else ''}{n} elements, got {t.numel()}")
    return t


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _check(rc, where):
    if rc != 0:
        raise JfnkError(rc, where)


class Context:
    """One grid / order / model; owns the library context."""

    def __init__(self, grid: Grid, k: int, phys: Physics, opts: Opts | None = None):
        h = C.c_void_p()
        _check(_lib().jfnk_create(C.byref(grid), k, C.byref(phys), C.byref(opts) if opts else None,
                                  C.byref(h)), "jfnk_create")
        self.h = h
        self.grid, self.k, self.phys, self.opts = grid, k, phys, opts
        self.N = _lib().jfnk_num_unknowns(h)
        self.shape = (4, grid.nz, grid.nx, k + 1, k + 1)

    def close(self):
        if getattr(self, "h", None):
            _lib().jfnk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def workspace_bytes(grid: Grid, k: int, opts: Opts | None = None) -> int:
        return _lib().jfnk_workspace_bytes(C.byref(grid), k, C.byref(opts) if opts else None)

    def node_coords(self):
        import numpy as np
        n = self.N // 4
        x = np.empty(n)
        z = np.empty(n)
        _check(_lib().jfnk_node_coords(self.h, x.ctypes.data_as(C.c_void_p), z.ctypes.data_as(C.c_void_p)),
               "jfnk_node_coords")
        return x, z

    def jfnk_init_state(self, theta_pert, U, stream=None):
        _vec(theta_pert, self.N // 4, "theta_pert")
        _vec(U, self.N, "U")
        _check(_lib().jfnk_init_state(self.h, _ptr(theta_pert), _ptr(U), _stream(stream)), "jfnk_init_state")

    def dg_residual(self, U, f, stream=None):
        self._states(U=U, f=f)
        _check(_lib().dg_residual(self.h, _ptr(U), _ptr(f), _stream(stream)), "dg_residual")

    def jv_product(self, U, fU, y, alpha_dt, eps, Jy, stream=None):
        self._states(U=U, fU=fU, y=y, Jy=Jy)
        _check(_lib().jv_product(self.h, _ptr(U), _ptr(fU), _ptr(y), float(alpha_dt), float(eps), _ptr(Jy),
                                 _stream(stream)), "jv_product")

    def mg_precondition(self, U, alpha_dt, r, z, stream=None):
        self._states(U=U, r=r, z=z)
        _check(_lib().mg_precondition(self.h, _ptr(U), float(alpha_dt), _ptr(r), _ptr(z), _stream(stream)),
               "mg_precondition")

    def implicit_step(self, U, dt, scheme=1, stream=None, raise_on_error=True) -> Stats:
        self._states(U=U)
        st = Stats()
        rc = _lib().implicit_step(self.h, _ptr(U), float(dt), int(scheme), C.byref(st), _stream(stream))
        if raise_on_error:
            _check(rc, "implicit_step")
        return st

    def norm2(self, x, out, n=None, stream=None):
        n = _check_norm_args(x, out, n)
        _check(_lib().jfnk_norm2(self.h, _ptr(x), n, _ptr(out), _stream(stream)), "jfnk_norm2")

    def eos_pressure(self, E, p, stream=None):
        _vec(E, 0, "E", at_least=True)
        _vec(p, E.numel(), "p", at_least=True)
        _check(_lib().jfnk_eos_pressure(self.h, _ptr(E), E.numel(), _ptr(p), _stream(stream)),
               "jfnk_eos_pressure")

    def tangent_product(self, U, y, adt, out, stream=None):
        self._states(U=U, y=y, out=out)
        _check(_lib().jfnk_tangent_product(self.h, _ptr(U), _ptr(y), float(adt), _ptr(out), _stream(stream)),
               "jfnk_tangent_product")

    def time_operator(self, which, U, y, reps, stream=None):
        self._states(U=U, y=y)
        ms = (C.c_double * 2)()
        _check(_lib().jfnk_time_operator(self.h, int(which), _ptr(U), _ptr(y), int(reps), ms, _stream(stream)),
               "jfnk_time_operator")
        return ms[0], ms[1]

    def _states(self, **arrays):
        """Every given array is a float64 state-sized vector (N elements)."""
        for name, t in arrays.items():
            _vec(t, self.N, name)

    def _fv_size(self, level):
        X, Z = C.c_int(), C.c_int()
        _check(_lib().jfnk_fv_level_size(self.h, int(level), C.byref(X), C.byref(Z)), "jfnk_fv_level_size")
        return 4 * X.value * Z.value

    def jfnk_autotune(self, U, y, reps=3, stream=None):
        self._states(U=U, y=y)
        best = (C.c_int * 4)()
        ms = (C.c_double * 2)()
        _check(_lib().jfnk_autotune(self.h, _ptr(U), _ptr(y), int(reps), best, ms, _stream(stream)),
               "jfnk_autotune")
        return {"tile_faces": best[0], "tile_volume": best[1], "tile_fv": best[2],
                "fv_split_cells": best[3], "dg_ms": ms[0], "precond_ms": ms[1]}

    def fv_levels(self):
        n = _lib().jfnk_fv_levels(self.h)
        out = []
        for l in range(n):
            X, Z = C.c_int(), C.c_int()
            _check(_lib().jfnk_fv_level_size(self.h, l, C.byref(X), C.byref(Z)), "jfnk_fv_level_size")
            out.append((X.value, Z.value))
        return out

    def transfer_to_fv(self, u, v, stream=None):
        self._states(u=u)
        _vec(v, self._fv_size(0), "v")
        _check(_lib().jfnk_transfer_to_fv(self.h, _ptr(u), _ptr(v), _stream(stream)), "jfnk_transfer_to_fv")

    def transfer_to_dg(self, v, u, stream=None):
        self._states(u=u)
        _vec(v, self._fv_size(0), "v")
        _check(_lib().jfnk_transfer_to_dg(self.h, _ptr(v), _ptr(u), _stream(stream)), "jfnk_transfer_to_dg")

    def fv_residual(self, level, u, f, stream=None):
        n = self._fv_size(level)
        _vec(u, n, "u")
        _vec(f, n, "f")
        _check(_lib().jfnk_fv_residual(self.h, int(level), _ptr(u), _ptr(f), _stream(stream)),
               "jfnk_fv_residual")
