"""Thin ctypes binding of libwcmg.so (include/wcmg.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Functions keep the C names; ``Context`` bundles a context handle with
the same calls for convenience.  Buffers may be numpy arrays (host memory,
complex128, C-contiguous) or torch CUDA tensors (device memory, complex128,
contiguous); the binding passes the pointer and the matching ``where`` flag.

Importing this module raises ImportError when the built library is missing:
there is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwcmg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "wcmg.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built: run paper_1904_08678_gb300/build.py (or __graft_entry__.build())")
_lib = ctypes.CDLL(LIB_PATH)

MAX_LEVELS = 4
NOALLOC_MAX_ELEMS = 262144
NKCLASS = 12
OK, ERR_ARG, ERR_CUDA, ERR_STATE, ERR_NOT_CONVERGED, ERR_NAN, ERR_TIMEOUT, ERR_OOM = 0, -1, -2, -3, -4, -5, -6, -7
F64, F32, BF16, F16 = 0, 1, 2, 3
HOST, DEVICE = 0, 1
KCLASS = ["dslash", "coarse", "restrict", "prolong", "blas", "ortho", "coarsen", "clover", "pack", "krylov",
          "dslash64", "ptc"]
PTC_HIDDEN, PTC_NWEIGHTS = 12, 3456
COARSE_MG, COARSE_WARMSTART, COARSE_LEARNED = 0, 1, 2
SMOOTHER_MR, SMOOTHER_GMRES, SMOOTHER_SAP = 0, 1, 2
NOPC = 5
OPC = ["apply", "restrict", "prolong", "ortho", "coarsen"]


class wcmg_params(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int * 4),
        ("n_levels", ctypes.c_int),
        ("block", (ctypes.c_int * 4) * (MAX_LEVELS - 1)),
        ("nvec", ctypes.c_int * (MAX_LEVELS - 1)),
        ("m0", ctypes.c_double),
        ("csw", ctypes.c_double),
        ("smoother_steps", ctypes.c_int),
        ("setup_init_sweeps", ctypes.c_int),
        ("setup_refine_sweeps", ctypes.c_int),
        ("coarse_restart", ctypes.c_int),
        ("coarse_maxiter", ctypes.c_int),
        ("coarse_tol", ctypes.c_double),
        ("outer_restart", ctypes.c_int),
        ("outer_maxiter", ctypes.c_int),
        ("outer_tol", ctypes.c_double),
        ("inner_prec", ctypes.c_int),
        ("coarse_link_prec", ctypes.c_int),
        ("max_rhs", ctypes.c_int),
        ("profile", ctypes.c_int),
        ("use_graphs", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("smoother", ctypes.c_int),
        ("kcycle", ctypes.c_int),
        ("kcycle_steps", ctypes.c_int),
        ("kcycle_tol", ctypes.c_double),
        ("sap_cycles", ctypes.c_int),
        ("sap_eo", ctypes.c_int),
        ("ortho_df", ctypes.c_int),
        ("coarse_eo", ctypes.c_int),
        ("coarse_sigma3", ctypes.c_int),
    ]


class wcmg_kstat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", ctypes.c_double), ("bytes", ctypes.c_double),
                ("flops", ctypes.c_double)]


class wcmg_stats(ctypes.Structure):
    _fields_ = [
        ("outer_iterations", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("true_residual", ctypes.c_double),
        ("coarse_iterations", ctypes.c_longlong),
        ("kernel_launches", ctypes.c_longlong),
        ("ms_setup_init", ctypes.c_double),
        ("ms_setup_refine", ctypes.c_double),
        ("ms_solve", ctypes.c_double),
        ("learned_fallback", ctypes.c_int),
        ("learned_cycles", ctypes.c_int),
        ("graph", ctypes.c_int),
        ("reserved", ctypes.c_int),
        ("k", wcmg_kstat * NKCLASS),
    ]

    def kernels(self):
        return {KCLASS[i]: dict(launches=self.k[i].launches, ms=self.k[i].ms, bytes=self.k[i].bytes,
                                flops=self.k[i].flops) for i in range(NKCLASS) if self.k[i].launches}


class wcmg_tile(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("rhs_per_cta", ctypes.c_int), ("parts", ctypes.c_int),
                ("threads", ctypes.c_int), ("ntile", ctypes.c_int), ("source", ctypes.c_int),
                ("candidates", ctypes.c_int), ("stages", ctypes.c_int), ("us", ctypes.c_double),
                ("us_default", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class wcmg_solve_opts(ctypes.Structure):
    _fields_ = [("zero_guess", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class wcmg_train_opts(ctypes.Structure):
    _fields_ = [("npairs", ctypes.c_int), ("batch", ctypes.c_int), ("steps", ctypes.c_int), ("refresh", ctypes.c_int),
                ("lr", ctypes.c_double), ("target_tol", ctypes.c_double), ("seed", ctypes.c_uint64)]


class wcmg_train_stats(ctypes.Structure):
    _fields_ = [("loss_initial", ctypes.c_double), ("loss_final", ctypes.c_double),
                ("ms_generate", ctypes.c_double), ("ms_train", ctypes.c_double),
                ("loss_heldout", ctypes.c_double), ("pairs_total", ctypes.c_longlong)]


_vp, _i, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_PCTX = ctypes.c_void_p
_SIGS = {
    "wcmg_default_params": ([ctypes.POINTER(wcmg_params)], _i),
    "wcmg_create": ([ctypes.POINTER(wcmg_params), ctypes.POINTER(_PCTX)], _i),
    "wcmg_destroy": ([_PCTX], None),
    "wcmg_last_error": ([_PCTX], ctypes.c_char_p),
    "wcmg_set_gauge": ([_PCTX, _vp, _i, _vp], _i),
    "wcmg_set_clover": ([_PCTX, _d, _vp], _i),
    "wcmg_set_clover_raw": ([_PCTX, _vp, _i, _vp], _i),
    "wcmg_get_clover": ([_PCTX, _vp, _i, _vp], _i),
    "wcmg_get_clover_inverse": ([_PCTX, _vp, _i, _vp], _i),
    "wcmg_apply_D": ([_PCTX, _vp, _vp, _i, _i, _i, _vp], _i),
    "wcmg_set_nullvecs": ([_PCTX, _i, _vp, _i, _vp], _i),
    "wcmg_get_nullvecs": ([_PCTX, _i, _vp, _i, _vp], _i),
    "wcmg_coarsen": ([_PCTX, _i, _vp], _i),
    "wcmg_get_coarse_links": ([_PCTX, _i, _vp, _i, _vp], _i),
    "wcmg_set_coarse_links": ([_PCTX, _i, _vp, _i, _vp], _i),
    "wcmg_restrict": ([_PCTX, _i, _vp, _vp, _i, _i, _i, _vp], _i),
    "wcmg_prolong": ([_PCTX, _i, _vp, _vp, _i, _i, _i, _vp], _i),
    "wcmg_apply_coarse": ([_PCTX, _i, _vp, _vp, _i, _i, _i, _vp], _i),
    "wcmg_setup": ([_PCTX, _vp, _i, _vp, ctypes.POINTER(wcmg_stats)], _i),
    "wcmg_setup_seeded": ([_PCTX, ctypes.c_ulonglong, _vp, ctypes.POINTER(wcmg_stats)], _i),
    "wcmg_mg_cycle": ([_PCTX, _vp, _vp, _i, _i, _vp], _i),
    "wcmg_krylov": ([_PCTX, _i, _i, _vp, _vp, _i, _i, _d, _i, _i, _vp, ctypes.POINTER(_i)], _i),
    "wcmg_solve": ([_PCTX, _vp, _vp, _i, _i, _vp, ctypes.POINTER(wcmg_stats)], _i),
    "wcmg_solve_ex": ([_PCTX, _vp, _vp, _i, ctypes.POINTER(wcmg_solve_opts), _i, _vp, ctypes.POINTER(wcmg_stats)],
                      _i),
    "wcmg_solve_batch": ([ctypes.POINTER(_PCTX), _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_i), _i,
                          _vp, ctypes.POINTER(wcmg_stats)], _i),
    "wcmg_set_profile": ([_PCTX, _i], _i),
    "wcmg_check_bounded_wait": ([_PCTX, ctypes.c_longlong, _vp], _i),
    "wcmg_get_coarse_tile": ([_PCTX, _i, _i, _i, ctypes.POINTER(wcmg_tile)], _i),
    "wcmg_tune_coarse": ([_PCTX, _i, _i, _i, _i, _vp, ctypes.POINTER(wcmg_tile)], _i),
    "wcmg_set_coarse_tile": ([_PCTX, _i, _i, _i, ctypes.POINTER(wcmg_tile)], _i),
    "wcmg_get_kstats": ([_PCTX, ctypes.POINTER(wcmg_kstat)], _i),
    "wcmg_get_opcounts": ([_PCTX, ctypes.POINTER(ctypes.c_longlong)], _i),
    "wcmg_block_orthonormalise_noalloc": ([_vp, _vp, ctypes.POINTER(_i), ctypes.POINTER(_i), _i, _vp], _i),
    "wcmg_ptc_set_weights": ([_PCTX, _vp, _i, _vp], _i),
    "wcmg_ptc_get_weights": ([_PCTX, _vp, _i, _vp], _i),
    "wcmg_ptc_forward": ([_PCTX, _vp, _vp, _i, _i, _vp], _i),
    "wcmg_ptc_backward": ([_PCTX, _vp, _vp, _vp, _vp, _i, _i, _vp], _i),
    "wcmg_ptc_train": ([_PCTX, ctypes.POINTER(wcmg_train_opts), ctypes.POINTER(wcmg_train_stats), _vp], _i),
    "wcmg_set_coarse_mode": ([_PCTX, _i, _d], _i),
    "wcmg_save_net": ([_PCTX, ctypes.c_char_p], _i),
    "wcmg_load_net": ([_PCTX, ctypes.c_char_p], _i),
    "wcmg_save_setup": ([_PCTX, ctypes.c_char_p], _i),
    "wcmg_load_setup": ([_PCTX, ctypes.c_char_p], _i),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res
    globals()[_name] = _f


def header_functions():
    """Names of the functions include/wcmg.h declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(wcmg_\w+)\s*\(", txt, re.M)))


def exported(name: str) -> bool:
    return hasattr(_lib, name)


class WcmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"wcmg error {code}: {msg}")
        self.code = code


def _buf(a, writable=False):
    """(pointer, where) of a numpy host array or a torch CUDA tensor (complex128)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.complex128 or not a.flags.c_contiguous:
            raise TypeError("host buffers must be C-contiguous complex128 numpy arrays")
        if writable and not a.flags.writeable:
            raise TypeError("output array is read-only")
        return a.ctypes.data, HOST
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous() or str(a.dtype) != "torch.complex128":
            raise TypeError("device buffers must be contiguous complex128 torch tensors")
        return a.data_ptr(), (DEVICE if a.is_cuda else HOST)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def default_params(**kw) -> wcmg_params:
    p = wcmg_params()
    wcmg_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("dims", "nvec"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = int(x)
        elif k == "blocks":
            for l, b in enumerate(v):
                for i, x in enumerate(b):
                    p.block[l][i] = int(x)
        else:
            setattr(p, k, v)
    return p


class Context:
    """Owns one wcmg_ctx; methods map one-to-one onto the C calls."""

    def __init__(self, params: wcmg_params):
        self.params = params
        h = _PCTX()
        rc = wcmg_create(ctypes.byref(params), ctypes.byref(h))
        if rc != OK:
            raise WcmgError(rc, "wcmg_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            wcmg_destroy(self.h)
            self.h = None

    __del__ = close

    def _check(self, rc, allow=()):
        if rc != OK and rc not in allow:
            raise WcmgError(rc, wcmg_last_error(self.h).decode())
        return rc

    def set_gauge(self, U, stream=None):
        p, w = _buf(U)
        return self._check(wcmg_set_gauge(self.h, p, w, _stream(stream)))

    def set_clover(self, csw, stream=None):
        return self._check(wcmg_set_clover(self.h, float(csw), _stream(stream)))

    def set_clover_raw(self, C, stream=None):
        p, w = _buf(C)
        return self._check(wcmg_set_clover_raw(self.h, p, w, _stream(stream)))

    def get_clover(self, C, stream=None):
        p, w = _buf(C, True)
        return self._check(wcmg_get_clover(self.h, p, w, _stream(stream)))

    def get_clover_inverse(self, C, stream=None):
        p, w = _buf(C, True)
        return self._check(wcmg_get_clover_inverse(self.h, p, w, _stream(stream)))

    def apply_D(self, inp, out, nrhs=1, prec=F64, stream=None):
        pi, wi = _buf(inp)
        po, wo = _buf(out, True)
        assert wi == wo
        return self._check(wcmg_apply_D(self.h, pi, po, nrhs, prec, wi, _stream(stream)))

    def set_nullvecs(self, level, vecs, stream=None):
        p, w = _buf(vecs)
        return self._check(wcmg_set_nullvecs(self.h, level, p, w, _stream(stream)))

    def get_nullvecs(self, level, vecs, stream=None):
        p, w = _buf(vecs, True)
        return self._check(wcmg_get_nullvecs(self.h, level, p, w, _stream(stream)))

    def coarsen(self, level, stream=None):
        return self._check(wcmg_coarsen(self.h, level, _stream(stream)))

    def get_coarse_links(self, level, A, stream=None):
        p, w = _buf(A, True)
        return self._check(wcmg_get_coarse_links(self.h, level, p, w, _stream(stream)))

    def set_coarse_links(self, level, A, stream=None):
        p, w = _buf(A)
        return self._check(wcmg_set_coarse_links(self.h, level, p, w, _stream(stream)))

    def restrict(self, level, fine, coarse, nrhs=1, prec=F64, stream=None):
        pi, wi = _buf(fine)
        po, wo = _buf(coarse, True)
        assert wi == wo
        return self._check(wcmg_restrict(self.h, level, pi, po, nrhs, prec, wi, _stream(stream)))

    def prolong(self, level, coarse, fine, nrhs=1, prec=F64, stream=None):
        pi, wi = _buf(coarse)
        po, wo = _buf(fine, True)
        assert wi == wo
        return self._check(wcmg_prolong(self.h, level, pi, po, nrhs, prec, wi, _stream(stream)))

    def apply_coarse(self, level, inp, out, nrhs=1, prec=F64, stream=None):
        pi, wi = _buf(inp)
        po, wo = _buf(out, True)
        assert wi == wo
        return self._check(wcmg_apply_coarse(self.h, level, pi, po, nrhs, prec, wi, _stream(stream)))

    def setup(self, init_vecs, stream=None):
        p, w = _buf(init_vecs)
        st = wcmg_stats()
        self._check(wcmg_setup(self.h, p, w, _stream(stream), ctypes.byref(st)))
        return st

    def setup_seeded(self, seed, stream=None):
        st = wcmg_stats()
        self._check(wcmg_setup_seeded(self.h, ctypes.c_ulonglong(seed % 2**64), _stream(stream), ctypes.byref(st)))
        return st

    def mg_cycle(self, r, e, nrhs=1, stream=None):
        pi, wi = _buf(r)
        po, wo = _buf(e, True)
        assert wi == wo
        return self._check(wcmg_mg_cycle(self.h, pi, po, nrhs, wi, _stream(stream)))

    def krylov(self, level, kind, b, x, nrhs=1, steps_or_restart=4, tol=0.0, maxiter=100, stream=None):
        pi, wi = _buf(b)
        po, wo = _buf(x, True)
        assert wi == wo
        its = ctypes.c_int(0)
        self._check(wcmg_krylov(self.h, level, kind, pi, po, nrhs, steps_or_restart, tol, maxiter, wi,
                                _stream(stream), ctypes.byref(its)))
        return its.value

    def solve(self, b, x, nrhs=1, stream=None, allow_not_converged=False):
        pi, wi = _buf(b)
        po, wo = _buf(x, True)
        assert wi == wo
        st = wcmg_stats()
        self._check(wcmg_solve(self.h, pi, po, nrhs, wi, _stream(stream), ctypes.byref(st)),
                    allow=(ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return st

    def solve_ex(self, b, x, nrhs=1, zero_guess=1, stream=None, allow_not_converged=False):
        """wcmg_solve_ex: zero_guess = 0 starts from the initial guess held in x."""
        pi, wi = _buf(b)
        po, wo = _buf(x, True)
        assert wi == wo
        o = wcmg_solve_opts(zero_guess=int(zero_guess))
        st = wcmg_stats()
        self._check(wcmg_solve_ex(self.h, pi, po, nrhs, ctypes.byref(o), wi, _stream(stream), ctypes.byref(st)),
                    allow=(ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return st

    def set_profile(self, mask):
        return self._check(wcmg_set_profile(self.h, mask))

    def check_bounded_wait(self, polls=1000, stream=None):
        """Return code of wcmg_check_bounded_wait (ERR_TIMEOUT when the bounded waits work)."""
        return self._check(wcmg_check_bounded_wait(self.h, int(polls), _stream(stream)), allow=(ERR_TIMEOUT,))

    def get_coarse_tile(self, level, nrhs=1, prec=F32):
        t = wcmg_tile()
        self._check(wcmg_get_coarse_tile(self.h, level, nrhs, prec, ctypes.byref(t)))
        return t.as_dict()

    def tune_coarse(self, level, nrhs=1, prec=F32, cold=0, stream=None):
        t = wcmg_tile()
        self._check(wcmg_tune_coarse(self.h, level, nrhs, prec, cold, _stream(stream), ctypes.byref(t)))
        return t.as_dict()

    def set_coarse_tile(self, level, nrhs=1, prec=F32, kind=-1, rhs_per_cta=0, parts=0, threads=0, ntile=0, stages=0):
        t = wcmg_tile(kind=kind, rhs_per_cta=rhs_per_cta, parts=parts, threads=threads, ntile=ntile, stages=stages)
        return self._check(wcmg_set_coarse_tile(self.h, level, nrhs, prec, ctypes.byref(t)))

    @staticmethod
    def solve_batch(ctxs, bs, xs, nrhs=None, stream=None, allow_not_converged=False):
        """wcmg_solve_batch over several contexts (one graph launch once warm)."""
        n = len(ctxs)
        nrhs = list(nrhs) if nrhs is not None else [1] * n
        hs = (_PCTX * n)(*[c.h for c in ctxs])
        pb, px, where = (_vp * n)(), (_vp * n)(), set()
        for i in range(n):
            pb[i], w1 = _buf(bs[i])
            px[i], w2 = _buf(xs[i], True)
            where |= {w1, w2}
        assert len(where) == 1
        sts = (wcmg_stats * n)()
        rc = wcmg_solve_batch(hs, n, pb, px, (_i * n)(*nrhs), where.pop(), _stream(stream), sts)
        if rc != OK and not (allow_not_converged and rc == ERR_NOT_CONVERGED):
            raise WcmgError(rc, wcmg_last_error(ctxs[0].h).decode())
        return list(sts)

    def kstats(self):
        arr = (wcmg_kstat * NKCLASS)()
        self._check(wcmg_get_kstats(self.h, arr))
        return {KCLASS[i]: dict(launches=arr[i].launches, ms=arr[i].ms, bytes=arr[i].bytes, flops=arr[i].flops)
                for i in range(NKCLASS)}

    def opcounts(self):
        """{kind: [count per level]} of wcmg_get_opcounts."""
        arr = (ctypes.c_longlong * (NOPC * MAX_LEVELS))()
        self._check(wcmg_get_opcounts(self.h, arr))
        return {k: [arr[i * MAX_LEVELS + l] for l in range(MAX_LEVELS)] for i, k in enumerate(OPC)}

    def ptc_set_weights(self, W, stream=None):
        p, w = _buf(W)
        return self._check(wcmg_ptc_set_weights(self.h, p, w, _stream(stream)))

    def ptc_get_weights(self, W, stream=None):
        p, w = _buf(W, True)
        return self._check(wcmg_ptc_get_weights(self.h, p, w, _stream(stream)))

    def ptc_forward(self, inp, out, nrhs=1, stream=None):
        pi, wi = _buf(inp)
        po, wo = _buf(out, True)
        assert wi == wo
        return self._check(wcmg_ptc_forward(self.h, pi, po, nrhs, wi, _stream(stream)))

    def ptc_backward(self, inp, gout, gin, gW, nrhs=1, stream=None):
        pi, wi = _buf(inp)
        pg, wg = _buf(gout)
        pgi, wgi = _buf(gin, True)
        pw, ww = _buf(gW, True)
        assert wi == wg == wgi == ww
        return self._check(wcmg_ptc_backward(self.h, pi, pg, pgi, pw, nrhs, wi, _stream(stream)))

    def ptc_train(self, npairs=32, batch=4, steps=100, lr=1e-3, target_tol=1e-6, seed=1, refresh=0, stream=None):
        o = wcmg_train_opts(npairs=npairs, batch=batch, steps=steps, refresh=refresh, lr=lr, target_tol=target_tol,
                            seed=seed)
        st = wcmg_train_stats()
        self._check(wcmg_ptc_train(self.h, ctypes.byref(o), ctypes.byref(st), _stream(stream)))
        return st

    def set_coarse_mode(self, mode, fallback_ratio=0.9):
        return self._check(wcmg_set_coarse_mode(self.h, mode, fallback_ratio))

    def save_net(self, path):
        return self._check(wcmg_save_net(self.h, path.encode()))

    def load_net(self, path):
        return self._check(wcmg_load_net(self.h, path.encode()))

    def save_setup(self, path):
        return self._check(wcmg_save_setup(self.h, path.encode()))

    def load_setup(self, path):
        return self._check(wcmg_load_setup(self.h, path.encode()))
