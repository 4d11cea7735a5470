"""Thin ctypes binding of libcombo.so (include/combo.h).

Argument marshalling only: every step of a solve runs in the CUDA library.
Host arrays are numpy arrays; device arrays are torch CUDA tensors (torch is
used only for device memory and streams).  There is no CPU fallback: if the
library is missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcombo.so")

OK, PENDING = 0, 1
E_NAMES = {-1: "invalid argument", -2: "out of memory", -3: "not converged", -4: "laminate Newton failed",
           -5: "inadmissible (det F <= 0)", -6: "NaN", -7: "timeout", -8: "CUDA error", -9: "cancelled"}
FP64, FP32_REFINED, FP32_REFINED_DF = 0, 1, 2
ROTATED, SPECTRAL, STAGGERED, STAGGERED_DFMG = 0, 1, 2, 3
FINITE_STRAIN, INFINITESIMAL_STRAIN = 0, 1
FIXED_POINT, NEWTON_CG, NONLINEAR_CG = 0, 1, 2
MEM_HOST, MEM_DEVICE = 0, 1


class ComboError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"combo error {code} ({E_NAMES.get(code, '?')}): {msg}")
        self.code = code


class CtxOpts(C.Structure):
    _fields_ = [("device", C.c_int32), ("stream", C.c_void_p)]


class ProblemS(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("l", C.c_double * 3), ("phase", C.c_void_p), ("n_boxels", C.c_int64),
                ("boxel_idx", C.c_void_p), ("boxel_N", C.c_void_p), ("boxel_c", C.c_void_p),
                ("mu", C.c_double * 2), ("lam", C.c_double * 2), ("Fbar", C.c_double * 9), ("n_steps", C.c_int32),
                ("mem", C.c_int32)]


class OptionsS(C.Structure):
    _fields_ = [("precision", C.c_int32), ("kspace", C.c_int32), ("solver", C.c_int32), ("tol", C.c_double),
                ("max_iter", C.c_int32), ("fixed_iterations", C.c_int32), ("cg_tol", C.c_double),
                ("cg_max_iter", C.c_int32), ("cg_fixed_iterations", C.c_int32), ("nr_tol_rel", C.c_double),
                ("nr_tol_abs", C.c_double), ("nr_max_iter", C.c_int32), ("c_min", C.c_double), ("mu0", C.c_double),
                ("theory", C.c_int32), ("wait_poll_cap", C.c_int32)]


class ResultS(C.Structure):
    _fields_ = [("Pbar", C.c_void_p), ("F_out", C.c_void_p), ("P_out", C.c_void_p), ("a_out", C.c_void_p),
                ("iters", C.c_void_p), ("cg_iters", C.c_void_p), ("resid", C.c_void_p), ("mem", C.c_int32),
                ("steps_done", C.c_int32), ("nr_iters", C.c_int64), ("n_backproj", C.c_int64),
                ("n_laminate_evals", C.c_int64), ("n_operator", C.c_int64), ("n_operator_fp64", C.c_int64),
                ("Pbar_phase", C.c_void_p)]


EXPORTS = ["combo_ctx_create", "combo_ctx_destroy", "combo_last_error", "combo_options_default",
           "combo_solve_footprint", "combo_solve", "combo_solve_begin", "combo_solve_advance", "combo_solve_advance_newton", "combo_solve_finish",
           "combo_solve_end", "combo_solve_batch", "combo_solve_profile", "combo_solve_profile_read", "combo_apply_G",
           "combo_constitutive", "combo_apply_G_noalloc", "combo_server_create", "combo_server_destroy",
           "combo_submit", "combo_poll", "combo_wait", "combo_cancel", "combo_server_stats",
           "combo_autotune_enable", "combo_autotune_force", "combo_autotune_report", "combo_coarse_grain",
           "combo_coarse_grain_profile", "combo_coarse_grain_profile_read", "combo_df_log", "combo_arith_rates",
           "combo_solve_advance_steps", "combo_state_export", "combo_state_import", "combo_neohooke_eval",
           "combo_laminate_eval", "combo_fault_inject_alloc", "combo_krylov_form"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libcombo.so (raises if it is missing; never falls back)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ComboError(-8, f"{path} is missing: build it with paper_2204_13624_gb300.build.build()")
    L = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    L.combo_ctx_create.argtypes = [vp, C.POINTER(vp)]
    L.combo_ctx_create.restype = C.c_int
    L.combo_ctx_destroy.argtypes = [vp]
    L.combo_last_error.restype = C.c_char_p
    L.combo_options_default.argtypes = [vp]
    L.combo_solve_footprint.argtypes = [vp, vp]
    L.combo_solve_footprint.restype = i64
    L.combo_solve.argtypes = [vp, vp, vp, vp]
    L.combo_solve.restype = C.c_int
    L.combo_solve_batch.argtypes = [vp, i32, vp, vp, vp]
    L.combo_solve_batch.restype = C.c_int
    L.combo_solve_begin.argtypes = [vp, vp, vp, C.POINTER(vp)]
    L.combo_solve_begin.restype = C.c_int
    L.combo_solve_advance.argtypes = [vp, i64]
    L.combo_solve_advance.restype = C.c_int
    L.combo_solve_advance_newton.argtypes = [vp, i64]
    L.combo_solve_advance_newton.restype = C.c_int
    L.combo_solve_finish.argtypes = [vp, vp]
    L.combo_solve_finish.restype = C.c_int
    L.combo_solve_end.argtypes = [vp]
    L.combo_solve_profile.argtypes = [vp, i32]
    L.combo_solve_profile.restype = C.c_int
    L.combo_solve_profile_read.argtypes = [vp, i32, vp, vp, vp]
    L.combo_solve_profile_read.restype = C.c_int
    L.combo_apply_G.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, i32]
    L.combo_apply_G.restype = C.c_int
    L.combo_constitutive.argtypes = [vp, vp, vp, vp, vp, vp, i32]
    L.combo_constitutive.restype = C.c_int
    L.combo_apply_G_noalloc.argtypes = [i32, vp, vp, vp, i32, vp, vp, vp]
    L.combo_apply_G_noalloc.restype = C.c_int
    L.combo_autotune_enable.argtypes = [i32]
    L.combo_autotune_enable.restype = None
    L.combo_krylov_form.argtypes = [i32]
    L.combo_krylov_form.restype = C.c_int
    L.combo_autotune_force.argtypes = [i32, i32]
    L.combo_autotune_force.restype = C.c_int
    L.combo_autotune_report.argtypes = [C.c_char_p, i64]
    L.combo_autotune_report.restype = i64
    L.combo_coarse_grain.argtypes = [vp, vp, vp, vp, i32, vp, vp, i64, vp, vp, vp, C.POINTER(i64), i32]
    L.combo_coarse_grain.restype = C.c_int
    L.combo_coarse_grain_profile.argtypes = [i32]
    L.combo_coarse_grain_profile.restype = C.c_int
    L.combo_coarse_grain_profile_read.argtypes = [vp]
    L.combo_coarse_grain_profile_read.restype = C.c_int
    L.combo_df_log.argtypes = [vp, vp, vp, C.c_int64]
    L.combo_df_log.restype = C.c_int
    L.combo_arith_rates.argtypes = [vp, vp]
    L.combo_arith_rates.restype = C.c_int
    L.combo_solve_advance_steps.argtypes = [vp, i32]
    L.combo_solve_advance_steps.restype = C.c_int
    L.combo_state_export.argtypes = [vp, vp, C.POINTER(C.c_int64)]
    L.combo_state_export.restype = C.c_int
    L.combo_state_import.argtypes = [vp, vp, C.c_int64]
    L.combo_state_import.restype = C.c_int
    L.combo_neohooke_eval.argtypes = [vp, vp, C.c_double, C.c_double, vp, vp]
    L.combo_neohooke_eval.restype = C.c_int
    L.combo_laminate_eval.argtypes = [vp, vp, vp, C.c_double, vp, vp, vp, vp, vp]
    L.combo_laminate_eval.restype = C.c_int
    L.combo_fault_inject_alloc.argtypes = [i64]
    L.combo_fault_inject_alloc.restype = C.c_int
    _lib = L
    return L


def _check(rc):
    if rc < 0:
        raise ComboError(rc, load().combo_last_error().decode())
    return rc


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _is_dev(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _torch_quiesce():
    """Wait for the work pending on torch's current stream before the library
    touches device memory torch allocated.  The library launches on its
    context's stream; torch's caching allocator orders reuse on torch's
    stream only, so a tensor handed out just now may sit in a block that a
    torch kernel still pending on that stream reads or writes."""
    import torch

    torch.cuda.current_stream().synchronize()


class Context:
    """A device, its stream and the library's memory (combo_ctx)."""

    def __init__(self, device: int = 0, stream=None):
        L = load()
        o = CtxOpts(device, stream)
        h = C.c_void_p()
        _check(L.combo_ctx_create(C.byref(o), C.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            load().combo_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx = None


def default_context() -> Context:
    global _default_ctx
    if _default_ctx is None:
        _default_ctx = Context(0)
    return _default_ctx


def options(**kw) -> OptionsS:
    o = OptionsS()
    load().combo_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Problem:
    """Marshals a problem dict (see microstructure.make_problem) into combo_problem.

    Arrays stay referenced by this object for the lifetime of the struct.
    Numpy arrays are host memory; torch CUDA tensors device memory."""

    def __init__(self, prob: dict):
        self.keep = []
        dev = _is_dev(prob["phase"])

        def arr(x, dt):
            if dev:
                return x.contiguous()
            return np.ascontiguousarray(x, dtype=dt)

        phase = arr(prob["phase"], np.uint8)
        bidx = arr(prob["boxel_idx"], np.int64)
        bN = arr(prob["boxel_N"], np.float64)
        bc = arr(prob["boxel_c"], np.float64)
        self.keep += [phase, bidx, bN, bc]
        s = ProblemS()
        s.n = (C.c_int32 * 3)(*[int(v) for v in prob["n"]])
        s.l = (C.c_double * 3)(*[float(v) for v in prob.get("l", (1.0, 1.0, 1.0))])
        s.phase = _ptr(phase)
        s.n_boxels = int(bidx.numel() if dev else bidx.size)
        s.boxel_idx = _ptr(bidx) if s.n_boxels else None
        s.boxel_N = _ptr(bN) if s.n_boxels else None
        s.boxel_c = _ptr(bc) if s.n_boxels else None
        s.mu = (C.c_double * 2)(*[float(v) for v in prob["mu"]])
        s.lam = (C.c_double * 2)(*[float(v) for v in prob["lam"]])
        s.Fbar = (C.c_double * 9)(*[float(v) for v in np.asarray(prob["Fbar"], dtype=np.float64).reshape(9)])
        s.n_steps = int(prob.get("n_steps", 1))
        s.mem = MEM_DEVICE if dev else MEM_HOST
        self.s = s
        self.n = tuple(int(v) for v in prob["n"])
        self.V = self.n[0] * self.n[1] * self.n[2]
        self.n_steps = s.n_steps
        self.n_boxels = s.n_boxels


def _result_buffers(pb: Problem, fields: bool, device: bool):
    S, V, nb = pb.n_steps, pb.V, pb.n_boxels
    out = dict(Pbar=np.zeros((S, 9)), iters=np.zeros(S, np.int32), cg_iters=np.zeros(S, np.int32),
               resid=np.zeros(S), Pbar_phase=np.zeros((S, 2, 9)))
    r = ResultS()
    r.Pbar = _ptr(out["Pbar"])
    r.Pbar_phase = _ptr(out["Pbar_phase"])
    r.iters = _ptr(out["iters"])
    r.cg_iters = _ptr(out["cg_iters"])
    r.resid = _ptr(out["resid"])
    if fields:
        if device:
            import torch

            out["F"] = torch.empty((9, V), dtype=torch.float64, device="cuda")
            out["P"] = torch.empty((9, V), dtype=torch.float64, device="cuda")
            out["a"] = torch.empty((max(nb, 1), 3), dtype=torch.float64, device="cuda")
            r.mem = MEM_DEVICE
            # Pbar etc. are host arrays; with mem = device the library expects
            # device pointers for every array, so keep scalars on the device too
            for k in ("Pbar", "iters", "cg_iters", "resid", "Pbar_phase"):
                out[k] = torch.as_tensor(out[k]).cuda()
            r.Pbar, r.iters, r.cg_iters, r.resid, r.Pbar_phase = (
                _ptr(out[k]) for k in ("Pbar", "iters", "cg_iters", "resid", "Pbar_phase"))
        else:
            out["F"] = np.zeros((9, V))
            out["P"] = np.zeros((9, V))
            out["a"] = np.zeros((max(nb, 1), 3))
            r.mem = MEM_HOST
        r.F_out = _ptr(out["F"])
        r.P_out = _ptr(out["P"])
        r.a_out = _ptr(out["a"])
    return out, r


def _collect(out, r, nb):
    out.update(steps_done=r.steps_done, nr_iters=r.nr_iters, n_backproj=r.n_backproj,
               n_laminate_evals=r.n_laminate_evals, n_operator=r.n_operator, n_operator_fp64=r.n_operator_fp64)
    if "a" in out:
        out["a"] = out["a"][:nb]
    return out


def solve(prob: dict, ctx: Context | None = None, fields: bool = True, device_results: bool = False, **opts):
    """combo_solve: full solve of every load step; returns Pbar per step,
    iteration counts, residuals, counters and (optionally) F, P, a."""
    ctx = ctx or default_context()
    pb = Problem(prob)
    o = options(**opts)
    out, r = _result_buffers(pb, fields, device_results)
    if device_results or pb.s.mem == MEM_DEVICE:
        _torch_quiesce()
    _check(load().combo_solve(ctx.h, C.byref(pb.s), C.byref(o), C.byref(r)))
    return _collect(out, r, pb.n_boxels)


def solve_record(prob: dict, result: dict, seconds: float | None = None, **opts) -> str:
    """One JSON line describing a finished solve: grid, boxels, options,
    load steps, per-step outer / CG iterations and residuals, Pbar per step,
    the laminate and operator counters, wall time if given, and the bytes of
    the fields a solve keeps resident (nine FP64 components of F and the
    spectrum).  Host-side formatting of a result dict returned by solve(),
    Solve.finish() or solve_batch()."""
    import json

    o = options(**opts)
    n = [int(v) for v in prob["n"]]
    V = n[0] * n[1] * n[2]
    nhp = (n[0] // 2 + 1 + 3) // 4 * 4
    rec = {"grid": n, "voxels": V, "boxels": int(len(prob.get("boxel_idx", []))),
           "precision": int(o.precision), "kspace": int(o.kspace), "solver": int(o.solver),
           "theory": int(o.theory), "tol": float(o.tol), "load_steps": int(result.get("steps_done", 0)),
           "outer_iterations": [int(v) for v in np.asarray(result["iters"]).ravel()],
           "cg_iterations": [int(v) for v in np.asarray(result.get("cg_iters", [])).ravel()],
           "residuals": [float(v) for v in np.asarray(result["resid"]).ravel()],
           "Pbar": np.asarray(result["Pbar"], dtype=float).reshape(-1, 9).tolist(),
           "nr_iterations": int(result.get("nr_iters", 0)), "back_projections": int(result.get("n_backproj", 0)),
           "laminate_evaluations": int(result.get("n_laminate_evals", 0)),
           "operator_applications": int(result.get("n_operator", 0)),
           "resident_field_bytes": 8 * 9 * V + 16 * 9 * n[2] * n[1] * nhp}
    if seconds is not None:
        rec["seconds"] = float(seconds)
    return json.dumps(rec)


def autotune_enable(enable: bool = True):
    load().combo_autotune_enable(1 if enable else 0)


KRYLOV_NINE, KRYLOV_DISPLACEMENT, KRYLOV_NODAL = 0, 1, 2


def krylov_form(form: int = KRYLOV_NODAL):
    """Most reduced evaluation form of the rotated operator that the FP32
    Krylov passes of solves set up afterwards may use (nine-component,
    displacement, nodal)."""
    _check(load().combo_krylov_form(int(form)))


def autotune_force(pass_index: int, candidate: int):
    """Force launch-shape candidate (0, 1) of pass 0..3 for solves set up
    afterwards; -1 returns to the tuned choice."""
    _check(load().combo_autotune_force(pass_index, candidate))


def autotune_report() -> str:
    n = load().combo_autotune_report(None, 0)
    buf = C.create_string_buffer(int(n) + 1)
    load().combo_autotune_report(buf, n + 1)
    return buf.value.decode()


def solve_batch(probs: list, ctx: Context | None = None, fields: bool = True, device_results: bool = False, **opts):
    """combo_solve_batch: independent problems on one grid solved together
    (stacked, one launch per pass for all of them); a list of results as
    from solve()."""
    ctx = ctx or default_context()
    pbs = [Problem(p) for p in probs]
    o = options(**opts)
    bufs = [_result_buffers(pb, fields, device_results) for pb in pbs]
    parr = (ProblemS * len(pbs))(*[pb.s for pb in pbs])
    rarr = (ResultS * len(pbs))(*[r for _, r in bufs])
    if device_results or any(pb.s.mem == MEM_DEVICE for pb in pbs):
        _torch_quiesce()
    _check(load().combo_solve_batch(ctx.h, len(pbs), C.byref(parr), C.byref(o), C.byref(rarr)))
    return [_collect(out, rarr[i], pbs[i].n_boxels) for i, (out, _) in enumerate(bufs)]


class Solve:
    """Incremental solve (combo_solve_begin / advance / finish / end)."""

    def __init__(self, prob: dict, ctx: Context | None = None, **opts):
        self.ctx = ctx or default_context()
        self.pb = Problem(prob)
        self.o = options(**opts)
        h = C.c_void_p()
        if self.pb.s.mem == MEM_DEVICE:
            _torch_quiesce()
        _check(load().combo_solve_begin(self.ctx.h, C.byref(self.pb.s), C.byref(self.o), C.byref(h)))
        self.h = h

    def advance(self, max_operator: int = 0) -> bool:
        """Run up to max_operator operator applications; True when finished."""
        return _check(load().combo_solve_advance(self.h, int(max_operator))) == OK

    def advance_newton(self, min_operator: int) -> bool:
        """Run at least min_operator operator applications and on to the end
        of the Newton step reached; True when finished."""
        return _check(load().combo_solve_advance_newton(self.h, int(min_operator))) == OK

    def finish(self, fields: bool = True, device_results: bool = False):
        out, r = _result_buffers(self.pb, fields, device_results)
        if device_results:
            _torch_quiesce()
        _check(load().combo_solve_finish(self.h, C.byref(r)))
        return _collect(out, r, self.pb.n_boxels)

    def advance_steps(self, k: int) -> bool:
        """Run k more load steps (stopping between steps); True when finished."""
        return _check(load().combo_solve_advance_steps(self.h, int(k))) == OK

    def export_state(self) -> bytes:
        """combo_state_export: the solve's state between load steps, as bytes."""
        n = C.c_int64(0)
        _check(load().combo_state_export(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(load().combo_state_export(self.h, buf, C.byref(n)))
        return buf.raw[: n.value]

    def import_state(self, blob: bytes):
        """combo_state_import into this solve (begun with the same problem and
        options, not yet advanced)."""
        buf = C.create_string_buffer(bytes(blob), len(blob))
        _check(load().combo_state_import(self.h, buf, len(blob)))

    def profile(self, enable: bool = True):
        """Start (reset) or stop per-kernel CUDA-event timing."""
        _check(load().combo_solve_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{kernel class: (total ms, launches)}"""
        n = 32
        names = C.create_string_buffer(32 * n)
        ms = np.zeros(n)
        cnt = np.zeros(n, np.int64)
        k = _check(load().combo_solve_profile_read(self.h, n, names, _ptr(ms), _ptr(cnt)))
        raw = names.raw
        out = {}
        for i in range(k):
            nm = raw[32 * i: 32 * i + 32].split(b"\0")[0].decode()
            out[nm] = (float(ms[i]), int(cnt[i]))
        return out

    def close(self):
        if self.h:
            load().combo_solve_end(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def footprint(prob: dict, **opts) -> int:
    pb = Problem(prob)
    o = options(**opts)
    return int(load().combo_solve_footprint(C.byref(pb.s), C.byref(o)))


def apply_G(X, n, l=(1.0, 1.0, 1.0), kspace=ROTATED, precision=FP64, ctx: Context | None = None):
    """Y = G[X] (mu0 Gamma0) of a real field X[9][V]; returns (Y, sum |Y|^2)."""
    ctx = ctx or default_context()
    dev = _is_dev(X)
    if dev:
        import torch

        X = X.contiguous().to(torch.float64)
        Y = torch.empty_like(X)
        _torch_quiesce()
    else:
        X = np.ascontiguousarray(X, dtype=np.float64)
        Y = np.zeros_like(X)
    nn = (C.c_int32 * 3)(*[int(v) for v in n])
    ll = (C.c_double * 3)(*[float(v) for v in l])
    ss = C.c_double(0.0)
    _check(load().combo_apply_G(ctx.h, nn, ll, kspace, precision, _ptr(X), _ptr(Y), C.byref(ss),
                                MEM_DEVICE if dev else MEM_HOST))
    return Y, ss.value


def constitutive(prob: dict, F, a=None, ctx: Context | None = None, **opts):
    """P[9][V] of a field F[9][V] (pure Neo-Hookean + boxel laminates); a is
    the [n_boxels][3] warm start, returned updated."""
    ctx = ctx or default_context()
    pb = Problem(prob)
    o = options(**opts)
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(9, -1)
    nb = pb.n_boxels
    a = np.zeros((max(nb, 1), 3)) if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1, 3).copy()
    P = np.zeros_like(F)
    _check(load().combo_constitutive(ctx.h, C.byref(pb.s), C.byref(o), _ptr(F), _ptr(a), _ptr(P), MEM_HOST))
    return P, a[:nb]


def neohooke_eval(F, mu, lam, ctx: Context | None = None):
    """combo_neohooke_eval: (P [9], A [9, 9]) of one Neo-Hookean phase at F."""
    ctx = ctx or default_context()
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(9)
    P, A = np.zeros(9), np.zeros(81)
    _check(load().combo_neohooke_eval(ctx.h, _ptr(F), float(mu), float(lam), _ptr(P), _ptr(A)))
    return P, A.reshape(9, 9)


def laminate_eval(F, N, c, mat, a0=None, ctx: Context | None = None):
    """combo_laminate_eval: one composite boxel; mat = (mu-, lam-, mu+, lam+).
    Returns dict(P, A, a, iters)."""
    ctx = ctx or default_context()
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(9)
    N = np.ascontiguousarray(N, dtype=np.float64).reshape(3)
    m = np.ascontiguousarray(mat, dtype=np.float64).reshape(4)
    a = np.zeros(3) if a0 is None else np.ascontiguousarray(a0, dtype=np.float64).reshape(3).copy()
    P, A = np.zeros(9), np.zeros(81)
    it = np.zeros(1, np.int32)
    _check(load().combo_laminate_eval(ctx.h, _ptr(F), _ptr(N), float(c), _ptr(m), _ptr(a), _ptr(P), _ptr(A),
                                      _ptr(it)))
    return dict(P=P, A=A.reshape(9, 9), a=a, iters=int(it[0]))


def fault_inject_alloc(after: int):
    """Test hook: the device allocation after `after` more successful ones
    fails as out of memory (then the hook disarms); after < 0 disarms it."""
    _check(load().combo_fault_inject_alloc(int(after)))


def arith_rates(ctx: Context | None = None):
    """combo_arith_rates: the device's FP64 and FP32 FMA throughput in
    TFLOP/s (dependent FMA chains timed with CUDA events)."""
    ctx = ctx or default_context()
    r = np.zeros(2)
    _check(load().combo_arith_rates(ctx.h, _ptr(r)))
    return float(r[0]), float(r[1])


def df_log(x, ctx: Context | None = None):
    """combo_df_log: ln x in the double-float arithmetic of the double-float
    forms (for accuracy tests); x a host array of positive doubles."""
    ctx = ctx or default_context()
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.zeros_like(x)
    _check(load().combo_df_log(ctx.h, _ptr(x), _ptr(y), x.size))
    return y


NORMAL_LAPLACE = 0
NORMAL_KABEL = 1


def coarse_grain(chi, b, h=(1.0, 1.0, 1.0), method="laplace", ctx: Context | None = None, cap=None):
    """combo_coarse_grain: composite boxels of a binary fine image (Sec. 5).

    chi is [n3][n2][n1] (x fastest), nonzero = inclusion: a numpy array (the
    call copies it to the device and returns numpy arrays) or a CUDA uint8
    tensor (the outputs are then CUDA tensors).  b = (b1, b2, b3) fine voxels
    per coarse voxel, h the fine voxel edges, method "laplace" (Sec. 5) or
    "kabel" (Eq. normal:kabel).  Returns (phase [nc3, nc2, nc1] uint8,
    boxel_idx int64 [k] increasing, c_plus [k], N [k, 3], n_boxels) with
    k = min(n_boxels, cap); cap limits the boxels written (default: every
    coarse voxel, so k = n_boxels)."""
    ctx = ctx or default_context()
    m = {"laplace": NORMAL_LAPLACE, "kabel": NORMAL_KABEL}[method]
    dev = _is_dev(chi)
    n3, n2, n1 = (int(v) for v in chi.shape)
    b1, b2, b3 = (int(v) for v in b)
    nc = (n3 // b3, n2 // b2, n1 // b1) if (n1 % b1 == 0 and n2 % b2 == 0 and n3 % b3 == 0) else (0, 0, 0)
    ncv = max(nc[0] * nc[1] * nc[2], 1)
    cap = ncv if cap is None else int(cap)
    if dev:
        import torch

        if chi.dtype != torch.uint8 or not chi.is_contiguous():
            chi = chi.contiguous().to(torch.uint8)
        kw = dict(device=chi.device)
        phase = torch.empty(ncv, dtype=torch.uint8, **kw)
        idx = torch.empty(max(cap, 1), dtype=torch.int64, **kw)
        N = torch.empty((max(cap, 1), 3), dtype=torch.float64, **kw)
        c = torch.empty(max(cap, 1), dtype=torch.float64, **kw)
        _torch_quiesce()
    else:
        chi = np.ascontiguousarray(chi, dtype=np.uint8)
        phase = np.empty(ncv, np.uint8)
        idx = np.empty(max(cap, 1), np.int64)
        N = np.empty((max(cap, 1), 3), np.float64)
        c = np.empty(max(cap, 1), np.float64)
    nn = (C.c_int32 * 3)(n1, n2, n3)
    bb = (C.c_int32 * 3)(b1, b2, b3)
    hh = (C.c_double * 3)(*[float(v) for v in h])
    nb = C.c_int64(0)
    _check(load().combo_coarse_grain(ctx.h, nn, bb, hh, m, _ptr(chi), _ptr(phase), cap, _ptr(idx), _ptr(N),
                                     _ptr(c), C.byref(nb), MEM_DEVICE if dev else MEM_HOST))
    k = min(nb.value, cap)
    return phase.reshape(nc), idx[:k], c[:k], N[:k], nb.value


def coarse_grain_profile(enable: bool = True):
    """Record CUDA events around the coarse-graining launches (benchmarks)."""
    _check(load().combo_coarse_grain_profile(1 if enable else 0))


def coarse_grain_profile_read():
    """(pack, slab pass, scan, scatter, finish) durations in ms of the last coarse_grain call."""
    ms = (C.c_double * 5)()
    _check(load().combo_coarse_grain_profile_read(ms))
    return tuple(ms)


def apply_G_noalloc(X, Y, n, l=(1.0, 1.0, 1.0), kspace=ROTATED, device=0, stream=None, want_sumsq=True):
    """combo_apply_G_noalloc: Y = G[X] in FP64 for callers that cannot
    allocate device memory.  X and Y are CUDA tensors [9][V] of float64
    owned by the caller (they may be the same tensor); the library's
    scratch is a fixed 4 MiB device array (grids up to 32^3).  Returns
    sum |Y|^2 (synchronising the stream) or None."""
    if not (_is_dev(X) and _is_dev(Y)):
        raise ComboError(-1, "apply_G_noalloc takes CUDA tensors")
    _torch_quiesce()
    nn = (C.c_int32 * 3)(*[int(v) for v in n])
    ll = (C.c_double * 3)(*[float(v) for v in l])
    ss = C.c_double(0.0)
    _check(load().combo_apply_G_noalloc(int(device), stream, nn, ll, int(kspace), _ptr(X), _ptr(Y),
                                        C.byref(ss) if want_sumsq else None))
    return ss.value if want_sumsq else None


class ServerOpts(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("hbm_budget_bytes", C.c_int64), ("keep_fields", C.c_int32),
                ("batch_max", C.c_int32), ("batch_max_voxels", C.c_int64)]


class ServingStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("queued", C.c_int64),
                ("running", C.c_int64), ("peak_running", C.c_int64), ("in_use_bytes", C.c_int64),
                ("budget_bytes", C.c_int64), ("p50_seconds", C.c_double), ("p99_seconds", C.c_double),
                ("mean_seconds", C.c_double), ("batches", C.c_int64), ("batched_requests", C.c_int64)]


def _server_lib():
    L = load()
    if not getattr(L, "_server_bound", False):
        vp, i64 = C.c_void_p, C.c_int64
        L.combo_server_create.argtypes = [vp, vp, C.POINTER(vp)]
        L.combo_server_create.restype = C.c_int
        L.combo_server_destroy.argtypes = [vp]
        L.combo_submit.argtypes = [vp, vp, vp, C.POINTER(i64)]
        L.combo_submit.restype = C.c_int
        L.combo_poll.argtypes = [vp, i64, vp]
        L.combo_poll.restype = C.c_int
        L.combo_wait.argtypes = [vp, i64, i64, vp]
        L.combo_wait.restype = C.c_int
        L.combo_cancel.argtypes = [vp, i64]
        L.combo_cancel.restype = C.c_int
        L.combo_server_stats.argtypes = [vp, vp]
        L.combo_server_stats.restype = C.c_int
        L._server_bound = True
    return L


class Server:
    """Request loop over many solves (combo_server_*): submit problems as they
    arrive, poll or wait for results; admitted solves run concurrently in
    worker slots on their own streams, admission bounded by device memory."""

    def __init__(self, ctx: Context | None = None, max_slots: int = 4, hbm_budget_bytes: int = 0,
                 keep_fields: bool = False, batch_max: int = 8, batch_max_voxels: int = 0):
        L = _server_lib()
        self.ctx = ctx or default_context()
        o = ServerOpts(max_slots, hbm_budget_bytes, 1 if keep_fields else 0, batch_max, batch_max_voxels)
        h = C.c_void_p()
        _check(L.combo_server_create(self.ctx.h, C.byref(o), C.byref(h)))
        self.h = h
        self.keep_fields = keep_fields
        self._meta = {}

    def submit(self, prob: dict, **opts) -> int:
        pb = Problem(prob)
        o = options(**opts)
        t = C.c_int64(0)
        _check(_server_lib().combo_submit(self.h, C.byref(pb.s), C.byref(o), C.byref(t)))
        self._meta[t.value] = (pb.n_steps, pb.V)
        return t.value

    def _buffers(self, ticket):
        S, V = self._meta[ticket]
        out = dict(Pbar=np.zeros((S, 9)), iters=np.zeros(S, np.int32), cg_iters=np.zeros(S, np.int32),
                   resid=np.zeros(S), Pbar_phase=np.zeros((S, 2, 9)))
        r = ResultS()
        r.Pbar, r.iters, r.cg_iters, r.resid, r.Pbar_phase = (
            _ptr(out[k]) for k in ("Pbar", "iters", "cg_iters", "resid", "Pbar_phase"))
        if self.keep_fields:
            out["F"] = np.zeros((9, V))
            out["P"] = np.zeros((9, V))
            r.F_out, r.P_out = _ptr(out["F"]), _ptr(out["P"])
        return out, r

    def _finish(self, ticket, out, r):
        del self._meta[ticket]
        out.update(steps_done=r.steps_done, nr_iters=r.nr_iters, n_backproj=r.n_backproj, n_operator=r.n_operator,
                   n_operator_fp64=r.n_operator_fp64)
        return out

    def poll(self, ticket: int):
        """None while the request runs, else its result dict (raises on failure)."""
        out, r = self._buffers(ticket)
        rc = _server_lib().combo_poll(self.h, ticket, C.byref(r))
        if rc == PENDING:
            return None
        if rc < 0:
            self._meta.pop(ticket, None)
            _check(rc)
        return self._finish(ticket, out, r)

    def wait(self, ticket: int, timeout_ms: int = -1):
        out, r = self._buffers(ticket)
        rc = _server_lib().combo_wait(self.h, ticket, int(timeout_ms), C.byref(r))
        if rc < 0:
            if rc != -7:
                self._meta.pop(ticket, None)
            _check(rc)
        return self._finish(ticket, out, r)

    def cancel(self, ticket: int):
        _check(_server_lib().combo_cancel(self.h, ticket))

    def stats(self) -> dict:
        st = ServingStats()
        _check(_server_lib().combo_server_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServingStats._fields_}

    def close(self):
        if self.h:
            _server_lib().combo_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
