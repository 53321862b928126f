"""Thin ctypes binding of the C ABI in ``include/mg.h`` (argument marshalling only).

Every step of the solver runs in the CUDA library ``libmg_gb300.so``; this
module only converts torch tensors (device memory, streams) into pointers and
sizes and turns status codes into exceptions. There is no fallback: if the
library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

MG_MAX_LEVELS = 4
MG_FP64, MG_FP32, MG_FP16 = 0, 1, 2

STATUS = {0: "MG_OK", 1: "MG_ERR_INVALID_ARG", 2: "MG_ERR_CUDA", 3: "MG_ERR_OOM", 4: "MG_ERR_NOT_CONVERGED",
          5: "MG_ERR_NAN", 6: "MG_ERR_UNSUPPORTED", 7: "MG_ERR_STATE", 8: "MG_ERR_TIMEOUT"}


class MGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class mg_geom(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("dims", ctypes.c_int * 4), ("Nc", ctypes.c_int)]


class mg_params(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("block", (ctypes.c_int * 4) * (MG_MAX_LEVELS - 1)),
                ("Nv", ctypes.c_int * (MG_MAX_LEVELS - 1)), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
                ("omega", ctypes.c_double), ("n_pass", ctypes.c_int), ("nu_setup", ctypes.c_int),
                ("gcr_restart", ctypes.c_int), ("max_iter", ctypes.c_int), ("coarsest_lu_max", ctypes.c_int),
                ("coarsest_tol", ctypes.c_double), ("coarsest_restart", ctypes.c_int),
                ("coarsest_max_iter", ctypes.c_int), ("precision", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("max_rhs", ctypes.c_int), ("chiral_split", ctypes.c_int)]


class mg_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("true_rel_residual", ctypes.c_double),
                ("level_apps", ctypes.c_longlong * MG_MAX_LEVELS), ("coarsest_iters", ctypes.c_longlong),
                ("ms", ctypes.c_double), ("graphs", ctypes.c_int), ("setup_s", ctypes.c_double),
                ("solve_s", ctypes.c_double), ("fine_D_apps", ctypes.c_longlong)]

    def as_dict(self):
        return dict(iters=self.iters, converged=bool(self.converged), true_rel_residual=self.true_rel_residual,
                    level_apps=list(self.level_apps), coarsest_iters=self.coarsest_iters, ms=self.ms,
                    graphs=bool(self.graphs), setup_s=self.setup_s, solve_s=self.solve_s,
                    fine_D_apps=self.fine_D_apps)


class mg_cg_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("fine_apps", ctypes.c_longlong), ("ms", ctypes.c_double)]

    def as_dict(self):
        return dict(iters=self.iters, converged=bool(self.converged), rel_residual=self.rel_residual,
                    fine_apps=self.fine_apps, ms=self.ms)


_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libmg_gb300.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("CUDA library libmg_gb300.so is missing")
    lib = ctypes.CDLL(path)
    P, I, D, VP = ctypes.POINTER, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    ctxp = ctypes.c_void_p
    sig = {
        "mg_default_params": (None, [P(mg_params)]),
        "mg_setup": (I, [P(ctxp), P(mg_geom), VP, D, P(mg_params), VP]),
        "mg_solve": (I, [ctxp, VP, VP, I, D, P(mg_stats)]),
        "mg_setup_batch": (I, [I, P(ctxp), P(mg_geom), P(VP), P(D), P(mg_params), VP]),
        "mg_save_setup": (I, [ctxp, ctypes.c_char_p]),
        "mg_load_setup": (I, [P(ctxp), ctypes.c_char_p, VP, VP]),
        "mg_context_info": (I, [ctxp, P(mg_geom), P(mg_params), P(D)]),
        "mg_nullnet_create": (I, [P(ctxp), I, I, I, ctypes.c_uint64]),
        "mg_nullnet_destroy": (None, [ctxp]),
        "mg_nullnet_weight_count": (ctypes.c_longlong, [ctxp]),
        "mg_nullnet_get_weights": (I, [ctxp, VP]),
        "mg_nullnet_set_weights": (I, [ctxp, VP]),
        "mg_nullnet_forward": (I, [ctxp, P(mg_geom), I, VP, P(ctypes.c_uint64), VP, VP]),
        "mg_nullnet_gradient": (I, [ctxp, P(mg_geom), I, VP, P(ctypes.c_uint64), VP, P(I), P(D), VP, VP]),
        "mg_nullnet_train": (I, [ctxp, P(mg_geom), I, VP, VP, P(I), I, I, D, ctypes.c_uint64, P(D), VP]),
        "mg_setup_learned": (I, [P(ctxp), P(mg_geom), VP, D, P(mg_params), ctxp, ctypes.c_uint64, I, D, I, P(I),
                                 P(D), VP]),
        "mg_convergence_rate": (I, [ctxp, I, ctypes.c_uint64, P(D)]),
        "mg_alu_peak": (I, [I, P(D), VP]),
        "mg_solve_multi": (I, [I, P(ctxp), P(I), P(VP), P(VP), D, P(mg_stats)]),
        "mg_half_convert": (I, [I, I, VP, VP, ctypes.c_longlong, VP]),
        "mg_solve_batch": (I, [ctxp, I, VP, VP, P(D), D, P(mg_stats)]),
        "mg_coarse_apply_mrhs": (I, [ctxp, I, I, VP, VP, I]),
        "mg_update_mass": (I, [ctxp, D]),
        "mg_clone": (I, [ctxp, D, VP, P(ctxp)]),
        "mg_destroy": (None, [ctxp]),
        "mg_last_error": (ctypes.c_char_p, []),
        "mg_dslash": (I, [P(mg_geom), VP, D, VP, VP, I, VP]),
        "mg_level_apply": (I, [ctxp, I, VP, VP]),
        "mg_restrict": (I, [ctxp, I, VP, VP]),
        "mg_prolong": (I, [ctxp, I, VP, VP]),
        "mg_vcycle": (I, [ctxp, VP, VP]),
        "mg_smooth": (I, [ctxp, I, VP, VP, I]),
        "mg_build_level": (I, [ctxp, I, VP]),
        "mg_get_null_vectors": (I, [ctxp, I, VP]),
        "mg_get_prolongator": (I, [ctxp, I, VP]),
        "mg_get_coarse_op": (I, [ctxp, I, VP]),
        "mg_level_size": (I, [ctxp, I, P(ctypes.c_longlong), P(I)]),
        "mg_kernel_launches": (ctypes.c_longlong, []),
        "mg_smooth_fine_noalloc": (I, [P(mg_geom), VP, D, VP, VP, I, D, VP]),
        "mg_coarsest_solve": (I, [ctxp, VP, VP, P(ctypes.c_longlong), P(D)]),
        "mg_selftest_barrier": (I, [I, VP]),
        "mg_autotune_report": (ctypes.c_size_t, [ctypes.c_char_p, ctypes.c_size_t]),
        "mg_cg_setup": (I, [P(ctxp), P(mg_geom), VP, D, P(mg_params), VP]),
        "mg_cg_solve": (I, [ctxp, VP, VP, D, I, I, P(mg_cg_stats)]),
        "mg_cg_get_coarse_op": (I, [ctxp, I, VP]),
        "mg_cg_destroy": (I, [ctxp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names of the C ABI entry points this binding expects."""
    return ["mg_default_params", "mg_setup", "mg_solve", "mg_update_mass", "mg_destroy", "mg_last_error",
            "mg_dslash", "mg_level_apply", "mg_restrict", "mg_prolong", "mg_vcycle", "mg_smooth", "mg_build_level",
            "mg_get_null_vectors", "mg_get_prolongator", "mg_get_coarse_op", "mg_level_size", "mg_kernel_launches",
            "mg_smooth_fine_noalloc", "mg_coarsest_solve", "mg_selftest_barrier", "mg_solve_batch",
            "mg_coarse_apply_mrhs", "mg_autotune_report", "mg_clone", "mg_setup_batch", "mg_save_setup",
            "mg_load_setup", "mg_context_info", "mg_nullnet_create", "mg_nullnet_destroy", "mg_nullnet_weight_count",
            "mg_nullnet_get_weights", "mg_nullnet_set_weights", "mg_nullnet_forward", "mg_nullnet_gradient",
            "mg_nullnet_train", "mg_setup_learned", "mg_convergence_rate", "mg_alu_peak", "mg_solve_multi",
            "mg_half_convert", "mg_cg_setup", "mg_cg_solve", "mg_cg_get_coarse_op", "mg_cg_destroy"]


def autotune_report() -> dict:
    """mg_autotune_report: {kernel/shape key: chosen launch variant} of the library's autotuner."""
    lib = load()
    n = lib.mg_autotune_report(None, 0)
    buf = ctypes.create_string_buffer(n + 1)
    lib.mg_autotune_report(buf, n + 1)
    out = {}
    for item in buf.value.decode().split(";"):
        if item:
            k, v = item.rsplit("=", 1)
            out[k] = int(v)
    return out


def _check(code: int):
    if code != 0:
        raise MGError(code, load().mg_last_error().decode())


def _ptr(t: torch.Tensor, dtype=None, numel=None) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def make_geom(dims, Nc: int = 1) -> mg_geom:
    g = mg_geom()
    g.d = len(dims)
    for i, L in enumerate(dims):
        g.dims[i] = int(L)
    g.Nc = Nc
    return g


def mg_default_params(**overrides) -> mg_params:
    """Library defaults, then ``overrides`` (blocks / Nv may be given as lists per level)."""
    p = mg_params()
    load().mg_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "blocks":
            for l, blk in enumerate(v):
                for i, b in enumerate(blk):
                    p.block[l][i] = int(b)
        elif k == "Nv":
            for l, n in enumerate(v):
                p.Nv[l] = int(n)
        else:
            setattr(p, k, v)
    return p


def mg_dslash(U: torch.Tensor, inp: torch.Tensor, out: torch.Tensor, m: float, dims, precision: int = MG_FP64,
              stream=None):
    """out = D(U) inp on the fine lattice (asynchronous on the stream). ``dims`` of length 2:
    U(1) in 2d (2 spins); of length 4: SU(3) in 4d (U[x][mu][3][3], psi[x][4][3])."""
    dt = torch.complex128 if precision == MG_FP64 else torch.complex64
    V = 1
    for L in dims:
        V *= int(L)
    four = len(dims) == 4
    g = make_geom(dims, Nc=3 if four else 1)
    nu, npsi = (36 * V, 12 * V) if four else (2 * V, 2 * V)
    _check(load().mg_dslash(ctypes.byref(g), _ptr(U, dt, nu), float(m), _ptr(inp, dt, npsi),
                            _ptr(out, dt, npsi), precision, _stream(stream)))


def half_spinor(nsites: int, device="cuda") -> torch.Tensor:
    """Buffer of a half-precision spinor field with per-site norms (12 bytes per site)."""
    return torch.empty(12 * nsites, dtype=torch.uint8, device=device)


def half_links(nsites: int, device="cuda") -> torch.Tensor:
    """Buffer of half-precision 2d links (8 bytes per site)."""
    return torch.empty(8 * nsites, dtype=torch.uint8, device=device)


def mg_half_convert(what: int, src: torch.Tensor, dst: torch.Tensor, nsites: int, stream=None):
    """mg_half_convert: 0 complex spinor -> half, 1 half -> complex spinor, 2 complex links -> half
    (the complex side complex128 or complex64)."""
    cplx = src if what in (0, 2) else dst
    prec = MG_FP64 if cplx.dtype == torch.complex128 else MG_FP32
    _check(load().mg_half_convert(int(what), prec, _ptr(src), _ptr(dst), int(nsites), _stream(stream)))


def mg_dslash_half(U_h: torch.Tensor, in_h: torch.Tensor, out_h: torch.Tensor, m: float, dims, stream=None):
    """out = D(U) in on half-precision fields (layouts of mg_half_convert), FP32 arithmetic."""
    V = int(dims[0]) * int(dims[1])
    if U_h.numel() != 8 * V or in_h.numel() != 12 * V or out_h.numel() != 12 * V:
        raise ValueError("half buffers of the wrong size")
    g = make_geom(dims)
    _check(load().mg_dslash(ctypes.byref(g), _ptr(U_h), float(m), _ptr(in_h), _ptr(out_h), MG_FP16,
                            _stream(stream)))


def mg_smooth_fine_noalloc(U: torch.Tensor, b: torch.Tensor, x: torch.Tensor, m: float, dims, nu: int,
                           omega: float = 0.8, stream=None):
    """x = nu MR iterations on D(U) x = b, with no device allocation (lattices up to 256 x 256)."""
    V = int(dims[0]) * int(dims[1])
    g = make_geom(dims)
    _check(load().mg_smooth_fine_noalloc(ctypes.byref(g), _ptr(U, torch.complex128, 2 * V), float(m),
                                         _ptr(b, torch.complex128, 2 * V), _ptr(x, torch.complex128, 2 * V),
                                         int(nu), float(omega), _stream(stream)))


def mg_selftest_barrier(missing_arrivals: int, stream=None):
    """Bounded grid-barrier self-test: raises MGError(MG_ERR_TIMEOUT) when an arrival is missing."""
    _check(load().mg_selftest_barrier(int(missing_arrivals), _stream(stream)))


def solve_multi(contexts, chis, psis, tol: float, nrhs=None, raise_on_fail: bool = True) -> list:
    """mg_solve_multi: psis[i] = D_i^{-1} chis[i] for every context (nrhs[i] vectors each, default 1),
    all outer loops in one graph launch; returns the stats of every vector, context by context."""
    n = len(contexts)
    if not (len(chis) == len(psis) == n) or n < 1:
        raise ValueError("one source and one solution array per context")
    nr = [1] * n if nrhs is None else [int(k) for k in nrhs]
    hs = (ctypes.c_void_p * n)(*[c._need().value if hasattr(c._need(), "value") else c._need() for c in contexts])
    cp = (ctypes.c_void_p * n)(*[_ptr(chis[i], torch.complex128, contexts[i].n0 * nr[i]).value for i in range(n)])
    pp = (ctypes.c_void_p * n)(*[_ptr(psis[i], torch.complex128, contexts[i].n0 * nr[i]).value for i in range(n)])
    na = (ctypes.c_int * n)(*nr)
    st = (mg_stats * sum(nr))()
    code = load().mg_solve_multi(n, hs, na, cp, pp, float(tol), st)
    if code != 0 and (raise_on_fail or code != 4):
        _check(code)
    return [st[i].as_dict() for i in range(sum(nr))]


def mg_alu_peak(precision: int, stream=None) -> float:
    """Measured FMA throughput (TFLOP/s) of the current GPU in FP64 (0) or FP32 (1)."""
    t = ctypes.c_double(0.0)
    _check(load().mg_alu_peak(int(precision), ctypes.byref(t), _stream(stream)))
    return float(t.value)


def mg_kernel_launches() -> int:
    return int(load().mg_kernel_launches())


class Context:
    """A set-up multigrid hierarchy (wraps mg_ctx*). Use ``Context.setup``."""

    def __init__(self, handle, dims, params, stream):
        self._h = handle
        self.dims = tuple(dims)
        self.params = params
        self.stream = stream
        self.volume = 1
        for L in dims:
            self.volume *= int(L)
        self.four = len(dims) == 4
        self.n0 = self.volume * (12 if self.four else 2)  # fine-level dofs

    @classmethod
    def setup(cls, U: torch.Tensor, m: float, dims, params: mg_params | None = None, stream=None) -> "Context":
        """mg_setup: adaptive setup of the hierarchy for D(U) with mass m (``dims`` of length 2:
        U(1) links U[x][mu]; of length 4: SU(3) links U[x][mu][3][3], two levels, chiral_split = 1)."""
        lib = load()
        p = params if params is not None else mg_default_params()
        four = len(dims) == 4
        g = make_geom(dims, Nc=3 if four else 1)
        V = 1
        for L in dims:
            V *= int(L)
        h = ctypes.c_void_p()
        s = _stream(stream)
        _check(lib.mg_setup(ctypes.byref(h), ctypes.byref(g), _ptr(U, torch.complex128, (36 if four else 2) * V),
                            float(m), ctypes.byref(p), s))
        return cls(h, dims, p, s)

    @classmethod
    def setup_batch(cls, Us, masses, dims_list, params_list, stream=None) -> list:
        """mg_setup_batch: the adaptive setups of several configurations (possibly of different
        sizes) at once, each as Context.setup would make it; returns one Context per configuration."""
        lib = load()
        n = len(Us)
        if not (len(masses) == len(dims_list) == len(params_list) == n) or n < 1:
            raise ValueError("one mass, geometry and parameter set per configuration")
        geoms = (mg_geom * n)()
        ptrs = (ctypes.c_void_p * n)()
        ms = (ctypes.c_double * n)(*[float(m) for m in masses])
        ps = (mg_params * n)(*params_list)
        for i, (U, dims) in enumerate(zip(Us, dims_list)):
            four = len(dims) == 4
            geoms[i] = make_geom(dims, Nc=3 if four else 1)
            V = 1
            for L in dims:
                V *= int(L)
            ptrs[i] = _ptr(U, torch.complex128, (36 if four else 2) * V)
        hs = (ctypes.c_void_p * n)()
        s = _stream(stream)
        _check(lib.mg_setup_batch(n, hs, geoms, ptrs, ms, ps, s))
        return [cls(ctypes.c_void_p(hs[i]), dims_list[i], params_list[i], s) for i in range(n)]

    @classmethod
    def load(cls, path: str, U: torch.Tensor, dims, stream=None) -> "Context":
        """mg_load_setup: a context rebuilt from a setup saved by Context.save, on the same links U."""
        four = len(dims) == 4
        V = 1
        for L in dims:
            V *= int(L)
        h = ctypes.c_void_p()
        s = _stream(stream)
        _check(load().mg_load_setup(ctypes.byref(h), os.fsencode(path), _ptr(U, torch.complex128,
                                                                               (36 if four else 2) * V), s))
        p = mg_params()
        g = mg_geom()
        m = ctypes.c_double()
        _check(load().mg_context_info(h, ctypes.byref(g), ctypes.byref(p), ctypes.byref(m)))
        ctx = cls(h, dims, p, s)
        ctx.mass = float(m.value)
        return ctx

    @classmethod
    def setup_learned(cls, U: torch.Tensor, m: float, dims, params, net: "NullNet", noise_seed: int = 1,
                      nu_refine: int = 0, max_rate: float = 1.0, rate_steps: int = 4, stream=None):
        """mg_setup_learned: a hierarchy whose level-0 vectors the network predicts (optionally refined
        by nu_refine MR iterations), judged by the measured convergence rate, with the plain setup as
        fallback. Returns (context, used_learned, rate)."""
        g = make_geom(dims)
        V = int(dims[0]) * int(dims[1])
        h = ctypes.c_void_p()
        used = ctypes.c_int(0)
        rate = ctypes.c_double(0.0)
        s = _stream(stream)
        _check(load().mg_setup_learned(ctypes.byref(h), ctypes.byref(g), _ptr(U, torch.complex128, 2 * V), float(m),
                                       ctypes.byref(params), net._need(), int(noise_seed), int(nu_refine),
                                       float(max_rate), int(rate_steps), ctypes.byref(used), ctypes.byref(rate), s))
        return cls(h, dims, params, s), bool(used.value), float(rate.value)

    def convergence_rate(self, steps: int = 4, seed: int = 1) -> float:
        """mg_convergence_rate: asymptotic factor of e <- e - V(D e)."""
        r = ctypes.c_double(0.0)
        _check(load().mg_convergence_rate(self._need(), int(steps), int(seed), ctypes.byref(r)))
        return float(r.value)

    def save(self, path: str):
        """mg_save_setup: write this context's near-null vectors (and what identifies them) to path."""
        _check(load().mg_save_setup(self._need(), os.fsencode(path)))

    def close(self):
        if self._h:
            load().mg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _need(self):
        if not self._h:
            raise RuntimeError("context is closed")
        return self._h

    def level_size(self, level: int):
        n = ctypes.c_longlong()
        k = ctypes.c_int()
        _check(load().mg_level_size(self._need(), level, ctypes.byref(n), ctypes.byref(k)))
        return int(n.value), int(k.value)

    def _numel(self, level: int) -> int:
        n, k = self.level_size(level)
        return n * k

    def solve(self, chi: torch.Tensor, psi: torch.Tensor, tol: float, raise_on_fail: bool = True) -> dict:
        """mg_solve: psi = D^{-1} chi to relative true residual tol; returns the stats."""
        st = mg_stats()
        n = self.n0
        code = load().mg_solve(self._need(), _ptr(chi, torch.complex128, n), _ptr(psi, torch.complex128, n),
                               1, float(tol), ctypes.byref(st))
        if code != 0 and (raise_on_fail or code != 4):
            _check(code)
        return st.as_dict()

    def solve_nrhs(self, chi: torch.Tensor, psi: torch.Tensor, tol: float, raise_on_fail: bool = True) -> list:
        """mg_solve with nrhs = chi.shape[0] right-hand sides at the context mass; stats per vector."""
        nrhs = int(chi.shape[0])
        n = self.n0 * nrhs
        st = (mg_stats * nrhs)()
        code = load().mg_solve(self._need(), _ptr(chi, torch.complex128, n), _ptr(psi, torch.complex128, n),
                               nrhs, float(tol), st)
        if code != 0 and (raise_on_fail or code != 4):
            _check(code)
        return [st[v].as_dict() for v in range(nrhs)]

    def solve_batch(self, chi: torch.Tensor, psi: torch.Tensor, tol: float, masses=None,
                    raise_on_fail: bool = True) -> list:
        """mg_solve_batch: psi[v] = D(m_v)^{-1} chi[v] for the nrhs = chi.shape[0] vectors
        (masses: one per vector, or None for the context mass); returns the stats per vector."""
        nrhs = int(chi.shape[0])
        n = self.n0 * nrhs
        st = (mg_stats * nrhs)()
        mp = None
        if masses is not None:
            if len(masses) != nrhs:
                raise ValueError("one mass per right-hand side")
            mp = (ctypes.c_double * nrhs)(*[float(m) for m in masses])
        code = load().mg_solve_batch(self._need(), nrhs, _ptr(chi, torch.complex128, n),
                                     _ptr(psi, torch.complex128, n), mp, float(tol), st)
        if code != 0 and (raise_on_fail or code != 4):
            _check(code)
        return [st[v].as_dict() for v in range(nrhs)]

    def coarse_apply_mrhs(self, level: int, inp: torch.Tensor, out: torch.Tensor, tensor_cores=True):
        """mg_coarse_apply_mrhs: out[n] = A_level inp[n] (complex64) on tensor cores (BF16 operands,
        FP32 sums) or, with tensor_cores=False, on CUDA cores in FP32; an int passes the C value
        (4d: 2 splits the vectors into BF16 hi + lo, 3 the operator as well)."""
        nrhs = int(inp.shape[0])
        n = self._numel(level) * nrhs
        mode = int(tensor_cores) if not isinstance(tensor_cores, bool) else (1 if tensor_cores else 0)
        _check(load().mg_coarse_apply_mrhs(self._need(), int(level), nrhs, _ptr(inp, torch.complex64, n),
                                           _ptr(out, torch.complex64, n), mode))

    def info(self) -> dict:
        """mg_context_info: the parameters as given at setup (precision included) and the mass."""
        p = mg_params()
        g = mg_geom()
        m = ctypes.c_double()
        _check(load().mg_context_info(self._need(), ctypes.byref(g), ctypes.byref(p), ctypes.byref(m)))
        return {"precision": int(p.precision), "levels": int(p.levels), "mass": float(m.value), "params": p}

    def update_mass(self, m: float):
        _check(load().mg_update_mass(self._need(), float(m)))

    def clone(self, m: float, stream=None) -> "Context":
        """mg_clone: a new context at mass m reusing this context's setup (Galerkin rebuilt)."""
        h = ctypes.c_void_p()
        s = _stream(stream)
        _check(load().mg_clone(self._need(), float(m), s, ctypes.byref(h)))
        return Context(h, self.dims, self.params, s)

    def level_apply(self, level: int, inp: torch.Tensor, out: torch.Tensor):
        n = self._numel(level)
        _check(load().mg_level_apply(self._need(), level, _ptr(inp, torch.complex128, n),
                                     _ptr(out, torch.complex128, n)))

    def restrict(self, level: int, fine: torch.Tensor, coarse: torch.Tensor):
        _check(load().mg_restrict(self._need(), level, _ptr(fine, torch.complex128, self._numel(level)),
                                  _ptr(coarse, torch.complex128, self._numel(level + 1))))

    def prolong(self, level: int, coarse: torch.Tensor, fine: torch.Tensor):
        _check(load().mg_prolong(self._need(), level, _ptr(coarse, torch.complex128, self._numel(level + 1)),
                                 _ptr(fine, torch.complex128, self._numel(level))))

    def vcycle(self, b: torch.Tensor, x: torch.Tensor):
        n = self._numel(0)
        _check(load().mg_vcycle(self._need(), _ptr(b, torch.complex128, n), _ptr(x, torch.complex128, n)))

    def coarsest_solve(self, b: torch.Tensor, x: torch.Tensor):
        """mg_coarsest_solve: x = A_c^{-1} b on the coarsest level; returns (iterations, device ms)."""
        n = self._numel(int(self.params.levels) - 1)
        it = ctypes.c_longlong(0)
        ms = ctypes.c_double(0.0)
        _check(load().mg_coarsest_solve(self._need(), _ptr(b, torch.complex128, n), _ptr(x, torch.complex128, n),
                                        ctypes.byref(it), ctypes.byref(ms)))
        return int(it.value), float(ms.value)

    def smooth(self, level: int, b: torch.Tensor, x: torch.Tensor, nu: int):
        n = self._numel(level)
        _check(load().mg_smooth(self._need(), level, _ptr(b, torch.complex128, n), _ptr(x, torch.complex128, n),
                                int(nu)))

    def build_level(self, level: int, vectors: torch.Tensor):
        nv = self.params.Nv[level]
        _check(load().mg_build_level(self._need(), level, _ptr(vectors, torch.complex128, nv * self._numel(level))))

    def null_vectors(self, level: int) -> torch.Tensor:
        nv = self.params.Nv[level]
        n, k = self.level_size(level)
        out = torch.empty((nv, n, k), dtype=torch.complex128, device="cuda")
        _check(load().mg_get_null_vectors(self._need(), level, _ptr(out)))
        return out

    def prolongator(self, level: int) -> torch.Tensor:
        """The columns of P_level as level vectors (2 Nv of them with the chirality split)."""
        nv = self.params.Nv[level] * (2 if self.four else 1)
        n, k = self.level_size(level)
        out = torch.empty((nv, n, k), dtype=torch.complex128, device="cuda")
        _check(load().mg_get_prolongator(self._need(), level, _ptr(out)))
        return out

    def coarse_op(self, level: int) -> torch.Tensor:
        n, k = self.level_size(level)
        out = torch.empty((n, 9 if self.four else 5, k, k), dtype=torch.complex128, device="cuda")
        _check(load().mg_get_coarse_op(self._need(), level, _ptr(out)))
        return out


class CgContext:
    """MG-preconditioned CG on the normal equations (wraps mg_cg_ctx*): the paper's own experiment."""

    def __init__(self, handle, dims, params, stream):
        self._h, self.dims, self.params, self.stream = handle, tuple(dims), params, stream
        self.volume = int(dims[0]) * int(dims[1])

    @classmethod
    def setup(cls, U: torch.Tensor, m: float, dims, params: mg_params, stream=None) -> "CgContext":
        """mg_cg_setup: the adaptive hierarchy for A = D^dagger D (2d U(1) links U[x][mu])."""
        g = make_geom(dims)
        h = ctypes.c_void_p()
        s = _stream(stream)
        V = int(dims[0]) * int(dims[1])
        _check(load().mg_cg_setup(ctypes.byref(h), ctypes.byref(g), _ptr(U, torch.complex128, 2 * V), float(m),
                                  ctypes.byref(params), s))
        return cls(h, dims, params, s)

    def _need(self):
        if self._h is None:
            raise MGError(1, "context closed")
        return self._h

    def solve(self, chi: torch.Tensor, psi: torch.Tensor, tol: float, max_iter: int = 100000,
              precondition: bool = True, raise_on_fail: bool = True) -> dict:
        """mg_cg_solve: psi = D^-1 chi through the normal equations by (MG-preconditioned) CG."""
        st = mg_cg_stats()
        n = 2 * self.volume
        code = load().mg_cg_solve(self._need(), _ptr(chi, torch.complex128, n), _ptr(psi, torch.complex128, n),
                                  float(tol), int(max_iter), 1 if precondition else 0, ctypes.byref(st))
        if raise_on_fail or code not in (0, 4):
            _check(code)
        return st.as_dict()

    def coarse_op(self, level: int, nsites: int, N: int) -> torch.Tensor:
        """mg_cg_get_coarse_op: the 9-point stencil of level `level` as [site][o][row][col]."""
        out = torch.empty((nsites, 9, N, N), dtype=torch.complex128, device="cuda")
        _check(load().mg_cg_get_coarse_op(self._need(), int(level), _ptr(out)))
        return out

    def close(self):
        if self._h is not None:
            load().mg_cg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NullNet:
    """The learned near-null network (wraps mg_nullnet*): 4 parallel-transport layers
    cin -> channels -> channels -> channels -> nv, complex FP32 weights, bf16 activations."""

    def __init__(self, cin: int = 8, channels: int = 16, nv: int = 8, seed: int = 20070704):
        h = ctypes.c_void_p()
        _check(load().mg_nullnet_create(ctypes.byref(h), int(cin), int(channels), int(nv), int(seed)))
        self._h = h
        self.cin, self.channels, self.nv = cin, channels, nv

    def _need(self):
        if not self._h:
            raise RuntimeError("network is destroyed")
        return self._h

    def close(self):
        if self._h:
            load().mg_nullnet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def weight_count(self) -> int:
        return int(load().mg_nullnet_weight_count(self._need()))

    def get_weights(self):
        import numpy as np
        out = np.empty(self.weight_count(), dtype=np.complex64)
        _check(load().mg_nullnet_get_weights(self._need(), out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_weights(self, w):
        import numpy as np
        w = np.ascontiguousarray(w, dtype=np.complex64)
        if w.size != self.weight_count():
            raise ValueError("wrong number of weights")
        _check(load().mg_nullnet_set_weights(self._need(), w.ctypes.data_as(ctypes.c_void_p)))

    @staticmethod
    def _seeds(seeds):
        return (ctypes.c_uint64 * len(seeds))(*[int(x) for x in seeds])

    def forward(self, U: torch.Tensor, dims, seeds, stream=None) -> torch.Tensor:
        """Network output complex64 [f][x][2 nv] for the fields U (complex128 [f][x][2])."""
        nf = len(seeds)
        V = int(dims[0]) * int(dims[1])
        g = make_geom(dims)
        out = torch.empty((nf, V, 2 * self.nv), dtype=torch.complex64, device=U.device)
        _check(load().mg_nullnet_forward(self._need(), ctypes.byref(g), nf, _ptr(U, torch.complex128, nf * 2 * V),
                                         self._seeds(seeds), _ptr(out), _stream(stream)))
        return out

    def gradient(self, U: torch.Tensor, dims, seeds, target: torch.Tensor, block, stream=None):
        """(loss, dloss/dW^* as complex64 [count]) against target complex128 [f][k][x][2]."""
        import numpy as np
        nf = len(seeds)
        V = int(dims[0]) * int(dims[1])
        g = make_geom(dims)
        blk = (ctypes.c_int * 2)(int(block[0]), int(block[1]))
        loss = ctypes.c_double(0.0)
        grad = np.empty(self.weight_count(), dtype=np.complex64)
        _check(load().mg_nullnet_gradient(self._need(), ctypes.byref(g), nf, _ptr(U, torch.complex128, nf * 2 * V),
                                          self._seeds(seeds), _ptr(target, torch.complex128, nf * self.nv * 2 * V),
                                          blk, ctypes.byref(loss), grad.ctypes.data_as(ctypes.c_void_p),
                                          _stream(stream)))
        return float(loss.value), grad

    def train(self, U: torch.Tensor, dims, target: torch.Tensor, block, steps: int, batch: int, lr: float,
              seed: int = 1, stream=None):
        """Adam steps on batches of fields; returns the loss of every step."""
        nf = int(U.shape[0])
        V = int(dims[0]) * int(dims[1])
        g = make_geom(dims)
        blk = (ctypes.c_int * 2)(int(block[0]), int(block[1]))
        losses = (ctypes.c_double * max(1, steps))()
        _check(load().mg_nullnet_train(self._need(), ctypes.byref(g), nf, _ptr(U, torch.complex128, nf * 2 * V),
                                       _ptr(target, torch.complex128, nf * self.nv * 2 * V), blk, int(steps),
                                       int(batch), float(lr), int(seed), losses, _stream(stream)))
        return [losses[i] for i in range(steps)]
