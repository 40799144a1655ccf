"""Python binding of the C ABI in include/bdg.h (argument marshalling only).

Device memory and streams come from PyTorch; every computation runs in the
CUDA library libbdg.so built from csrc/.  If the library is missing the
import of this module still works but every call raises RuntimeError --
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libbdg.so")

OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_NAN, \
    ERR_UNSUPPORTED = range(9)
FP64, MIXED = 0, 1
C128, C64 = 0, 1
UV, FG = 0, 1
GRAM_SIMT, GRAM_TENSOR = 0, 1

STATUS_NAMES = {0: "BDG_OK", 1: "BDG_ERR_INVALID", 2: "BDG_ERR_NOMEM", 3: "BDG_ERR_CUDA",
                4: "BDG_ERR_BREAKDOWN", 5: "BDG_ERR_NOT_CONVERGED", 6: "BDG_ERR_TIMEOUT",
                7: "BDG_ERR_NAN", 8: "BDG_ERR_UNSUPPORTED"}

# every symbol include/bdg.h declares
EXPORTS = ("bdg_plan_create", "bdg_plan_destroy", "bdg_plan_mu", "bdg_apply", "bdg_biortho",
           "bdg_solve", "bdg_solve_batched", "bdg_get_solve_stats", "bdg_ground_state",
           "bdg_chemical_potentials_noalloc", "bdg_perturbed_density", "bdg_gram",
           "bdg_last_error")


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("beta_n", ctypes.c_double), ("beta_s", ctypes.c_double),
                ("p", ctypes.c_double), ("q", ctypes.c_double),
                ("mu", ctypes.c_double * 3), ("prec", ctypes.c_int), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("seed", ctypes.c_ulonglong), ("flags", ctypes.c_int)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("iterations_fp32", ctypes.c_int),
                ("applies_fp32", ctypes.c_int), ("applies_fp64", ctypes.c_int),
                ("seconds", ctypes.c_double), ("flops_update_df", ctypes.c_double)]


class BdgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load() -> ctypes.CDLL:
    """Load libbdg.so (built in-tree); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBPATH):
        raise RuntimeError(f"{LIBPATH} is missing: build it with paper_2506_08308_gb300.build.build()")
    lib = ctypes.CDLL(LIBPATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    lib.bdg_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Params), dp, dp, vp]
    lib.bdg_plan_destroy.argtypes = [vp]
    lib.bdg_plan_mu.argtypes = [vp, dp]
    lib.bdg_apply.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int, vp]
    lib.bdg_biortho.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, vp, vp, ctypes.c_int, ip, vp]
    lib.bdg_solve.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, dp, vp, dp, ip, vp]
    pp = ctypes.POINTER(ctypes.c_void_p)
    dpp = ctypes.POINTER(ctypes.POINTER(ctypes.c_double))
    lib.bdg_solve_batched.argtypes = [pp, ctypes.c_int, ip, ip, dpp, pp, dpp, ip, vp]
    lib.bdg_get_solve_stats.argtypes = [vp, ctypes.POINTER(SolveStats)]
    lib.bdg_ground_state.argtypes = [ctypes.POINTER(Params), ctypes.c_double, dp, dp, ctypes.c_double,
                                     ctypes.c_int, dp, dp, dp, ip, vp]
    lib.bdg_chemical_potentials_noalloc.argtypes = [vp, dp, vp]
    lib.bdg_perturbed_density.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, dp, dp, ctypes.c_int,
                                          ctypes.c_double, vp, vp]
    lib.bdg_gram.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_longlong, ctypes.c_int, vp,
                             ctypes.c_longlong, ctypes.c_int, ctypes.c_longlong, vp, vp]
    lib.bdg_last_error.argtypes = [vp]
    lib.bdg_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "bdg_last_error":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _stream_handle(stream) -> ctypes.c_void_p:
    """The cudaStream_t of a torch stream; None -> torch's current stream
    (NULL, the legacy default stream, when torch sees no CUDA device)."""
    import torch
    if stream is None:
        if not torch.cuda.is_available():
            return ctypes.c_void_p(None)
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(None)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check_out(out, shape, dtype, device):
    """A caller-supplied output tensor must match exactly: the library writes
    prod(shape) elements of dtype through its pointer and cannot see its size."""
    if (tuple(out.shape) != tuple(shape) or out.dtype != dtype or out.device != device
            or not out.is_contiguous()):
        raise ValueError(f"out must be a contiguous {dtype} tensor of shape {tuple(shape)} on {device}, "
                         f"got {out.dtype} {tuple(out.shape)} on {out.device}")


def make_params(n: Sequence[int], lo: Sequence[float], hi: Sequence[float], beta_n: float,
                beta_s: float, p: float = 0.0, q: float = 0.0, mu=None, prec: int = FP64,
                tol: float = 1e-10, maxit: int = 500, seed: int = 1) -> Params:
    prm = Params()
    prm.dim = len(n)
    for a in range(3):
        prm.n[a] = int(n[a]) if a < len(n) else 1
        prm.lo[a] = float(lo[a]) if a < len(n) else 0.0
        prm.hi[a] = float(hi[a]) if a < len(n) else 1.0
    prm.beta_n, prm.beta_s, prm.p, prm.q = float(beta_n), float(beta_s), float(p), float(q)
    for j in range(3):
        prm.mu[j] = math.nan if mu is None else float(mu[j])
    prm.prec, prm.tol, prm.maxit, prm.seed, prm.flags = int(prec), float(tol), int(maxit), int(seed), 0
    return prm


def params_from(w, **kw) -> Params:
    """Params from any object with the fields n, lo, hi, beta_n, beta_s, p, q."""
    return make_params(w.n, w.lo, w.hi, w.beta_n, w.beta_s, w.p, w.q, **kw)


def _check(lib, st: int, plan=None):
    if st != OK:
        msg = lib.bdg_last_error(plan if plan is not None else None)
        raise BdgError(st, msg.decode() if msg else "")


class Plan:
    """One BdG problem on the current CUDA device (bdg_plan_create)."""

    def __init__(self, prm: Params, V: np.ndarray, phi: np.ndarray, stream=None):
        self.lib = load()
        self.prm = prm
        self.npts = int(np.prod([prm.n[a] for a in range(prm.dim)]))
        V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        if V.size != self.npts or phi.size != 3 * self.npts:
            raise ValueError("V must have N_p and phi 3*N_p entries")
        h = ctypes.c_void_p()
        st = self.lib.bdg_plan_create(ctypes.byref(h), ctypes.byref(prm), _dptr(V), _dptr(phi),
                                      _stream_handle(stream))
        _check(self.lib, st)
        self.handle = h
        import torch
        # the library records the current device at creation; outputs the
        # binding allocates go there too
        self.device = torch.device("cuda", torch.cuda.current_device())

    @classmethod
    def from_workload(cls, w, V, phi, **kw):
        return cls(params_from(w, **kw), V, phi)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.bdg_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def mu(self) -> np.ndarray:
        out = np.zeros(3)
        _check(self.lib, self.lib.bdg_plan_mu(self.handle, _dptr(out)), self.handle)
        return out

    def chemical_potentials_noalloc(self, stream=None) -> np.ndarray:
        """bdg_chemical_potentials_noalloc: eq. chem-formula mu of the plan's Phi,
        computed without any device allocation (fixed library-owned scratch;
        grids of at most 16384 points; overlapping calls race)."""
        out = np.zeros(3)
        st = self.lib.bdg_chemical_potentials_noalloc(self.handle, _dptr(out), _stream_handle(stream))
        _check(self.lib, st, self.handle)
        return out

    def apply(self, x, mode: int = UV, out=None, stream=None):
        """y = M x for a CUDA tensor x of shape (nvec, 6, N_p), complex64/128."""
        import torch
        if not x.is_cuda or x.dim() != 3 or x.shape[1] != 6 or x.shape[2] != self.npts:
            raise ValueError("x must be a CUDA tensor of shape (nvec, 6, N_p)")
        dt = {torch.complex128: C128, torch.complex64: C64}.get(x.dtype)
        if dt is None:
            raise ValueError("x must be complex64 or complex128")
        x = x.contiguous()
        if out is None:
            out = torch.empty_like(x)
        _check_out(out, x.shape, x.dtype, x.device)
        st = self.lib.bdg_apply(self.handle, int(mode), dt, _ptr(x), _ptr(out), int(x.shape[0]),
                                _stream_handle(stream))
        _check(self.lib, st, self.handle)
        return out

    def perturbed_density(self, UV, omega, times, eps: float, out=None, stream=None):
        """bdg_perturbed_density: n[l, t, j, x] = |phi_j + eps (u_j^l e^{-i w_l t} +
        conj(v_j^l) e^{i w_l t})|^2 for a CUDA tensor UV of shape (nmode, 6, N_p)
        (complex128 -> float64 result, complex64 -> float32), shape
        (nmode, nt, 3, N_p)."""
        import torch
        if not UV.is_cuda or UV.dim() != 3 or UV.shape[1] != 6 or UV.shape[2] != self.npts:
            raise ValueError("UV must be a CUDA tensor of shape (nmode, 6, N_p)")
        dt = {torch.complex128: C128, torch.complex64: C64}.get(UV.dtype)
        if dt is None:
            raise ValueError("UV must be complex64 or complex128")
        UV = UV.contiguous()
        nmode = int(UV.shape[0])
        om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).reshape(-1))
        ts = np.ascontiguousarray(np.asarray(times, dtype=np.float64).reshape(-1))
        if om.size != nmode:
            raise ValueError("omega needs one value per mode")
        rdt = torch.float64 if dt == C128 else torch.float32
        if out is None:
            out = torch.empty((nmode, ts.size, 3, self.npts), device=UV.device, dtype=rdt)
        _check_out(out, (nmode, ts.size, 3, self.npts), rdt, UV.device)
        st = self.lib.bdg_perturbed_density(self.handle, dt, _ptr(UV), nmode, _dptr(om), _dptr(ts), int(ts.size),
                                            float(eps), _ptr(out), _stream_handle(stream))
        _check(self.lib, st, self.handle)
        return out

    def biortho(self, F, G, Fl=None, Gl=None, stream=None):
        """In-place bi-orthonormalization of F, G (CUDA, (ncol, 3, N_p) complex);
        returns the rank kept."""
        import torch
        if (Fl is None) != (Gl is None):
            raise ValueError("Fl and Gl go together: give both or neither")
        dt = {torch.complex128: C128, torch.complex64: C64}.get(F.dtype)
        if dt is None or not F.is_cuda or F.dim() != 3:
            raise ValueError("F must be a complex64/complex128 CUDA tensor of shape (ncol, 3, N_p)")
        shape = (int(F.shape[0]), 3, self.npts)
        _check_out(F, shape, F.dtype, F.device)      # updated in place: exact shape, contiguous
        _check_out(G, shape, F.dtype, F.device)
        nlock = 0 if Fl is None else int(Fl.shape[0])
        if nlock:
            _check_out(Fl, (nlock, 3, self.npts), F.dtype, F.device)
            _check_out(Gl, (nlock, 3, self.npts), F.dtype, F.device)
        rank = ctypes.c_int(0)
        st = self.lib.bdg_biortho(self.handle, dt, _ptr(F), _ptr(G), int(F.shape[0]), _ptr(Fl),
                                  _ptr(Gl), nlock, ctypes.byref(rank), _stream_handle(stream))
        _check(self.lib, st, self.handle)
        return rank.value

    def solve(self, k: int, m: int, X0=None, want_vectors: bool = True, stream=None,
              allow_not_converged: bool = False):
        """(omega[k], UV (k,6,N_p) complex128 CUDA tensor or None, resid[k], nconv)."""
        import torch
        omega = np.zeros(k)
        resid = np.zeros(k)
        nconv = ctypes.c_int(0)
        if X0 is not None:
            if not X0.is_cuda or X0.device != self.device:
                raise ValueError("X0 must be a CUDA tensor on the plan's device")
            _check_out(X0, (m, 6, self.npts), torch.complex128, X0.device)
        UVt = torch.empty((k, 6, self.npts), dtype=torch.complex128, device=self.device) if want_vectors else None
        st = self.lib.bdg_solve(self.handle, int(k), int(m), _ptr(X0), _dptr(omega), _ptr(UVt),
                                _dptr(resid), ctypes.byref(nconv), _stream_handle(stream))
        if not (allow_not_converged and st == ERR_NOT_CONVERGED):
            _check(self.lib, st, self.handle)
        return omega, UVt, resid, nconv.value

    def stats(self) -> dict:
        s = SolveStats()
        _check(self.lib, self.lib.bdg_get_solve_stats(self.handle, ctypes.byref(s)), self.handle)
        return {f: getattr(s, f) for f, _ in SolveStats._fields_}


def gram(A, B, engine: int = GRAM_TENSOR, out=None, stream=None):
    """bdg_gram: G = A^T B over real columns of two blocks of complex columns
    (torch complex64 or complex128 tensors of shape (ncol, n), contiguous
    rows, same dtype and device); G has shape (2 ncol_a, 2 ncol_b), FP64."""
    import torch
    lib = load()
    if A.dtype != B.dtype or A.dtype not in (torch.complex64, torch.complex128):
        raise ValueError("A and B must both be complex64 or both complex128")
    if A.dim() != 2 or B.dim() != 2 or A.shape[1] != B.shape[1]:
        raise ValueError("A and B must be (ncol, n) with the same n")
    if A.device != B.device or A.device.type != "cuda":
        raise ValueError("A and B must be CUDA tensors on one device")
    if A.stride(1) != 1 or B.stride(1) != 1:
        raise ValueError("rows of A and B must be contiguous")
    shape = (2 * A.shape[0], 2 * B.shape[0])
    if out is None:
        out = torch.empty(shape, dtype=torch.float64, device=A.device)
    else:
        _check_out(out, shape, torch.float64, A.device)
    dtype = C64 if A.dtype == torch.complex64 else C128
    st = lib.bdg_gram(dtype, int(engine), _ptr(A), A.stride(0), A.shape[0], _ptr(B), B.stride(0), B.shape[0],
                      A.shape[1], _ptr(out), _stream_handle(stream))
    _check(lib, st)
    return out


def solve_batched(plans, ks, ms, want_vectors: bool = True, stream=None, allow_not_converged: bool = False):
    """bdg_solve_batched over independent plans: a list of (omega, UV or None,
    resid, nconv) per plan."""
    import torch
    lib = load()
    n = len(plans)
    dptr_t = ctypes.POINTER(ctypes.c_double)
    oms = [np.zeros(k) for k in ks]
    res = [np.zeros(k) for k in ks]
    uvs = [torch.empty((k, 6, p.npts), dtype=torch.complex128, device=p.device) if want_vectors else None
           for k, p in zip(ks, plans)]
    h = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    karr = (ctypes.c_int * n)(*ks)
    marr = (ctypes.c_int * n)(*ms)
    oarr = (dptr_t * n)(*[_dptr(o) for o in oms])
    rarr = (dptr_t * n)(*[_dptr(r) for r in res])
    uarr = (ctypes.c_void_p * n)(*[(u.data_ptr() if u is not None else None) for u in uvs])
    nconv = (ctypes.c_int * n)()
    st = lib.bdg_solve_batched(h, n, karr, marr, oarr, uarr, rarr, nconv, _stream_handle(stream))
    if not (allow_not_converged and st == ERR_NOT_CONVERGED):
        _check(lib, st)
    return [(oms[i], uvs[i], res[i], nconv[i]) for i in range(n)]


def ground_state(prm: Params, M: float, V: np.ndarray, phi0: np.ndarray, tol: float = 1e-12,
                 maxit: int = 200000, stream=None):
    """bdg_ground_state: (phi (3,N_p), mu[3], residual, iterations), on the GPU."""
    lib = load()
    npts = int(np.prod([prm.n[a] for a in range(prm.dim)]))
    V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(-1)
    phi = np.zeros(3 * npts)
    mu = np.zeros(3)
    res = np.zeros(1)
    it = ctypes.c_int(0)
    st = lib.bdg_ground_state(ctypes.byref(prm), float(M), _dptr(V), _dptr(phi0), float(tol), int(maxit),
                              _dptr(phi), _dptr(mu), _dptr(res), ctypes.byref(it), _stream_handle(stream))
    _check(lib, st)
    return phi.reshape(3, npts), mu, float(res[0]), it.value
