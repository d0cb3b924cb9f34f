"""Python binding of libeacg: the eARCG Kohn-Sham minimisation (arXiv 2503.16225) on a GB300.

Argument marshalling only: every step of the computation runs in the CUDA kernels of
libeacg.so (built in-tree by ``paper_2503_16225_gb300.build``).  The functions keep the C
names of ``include/eacg.h``; tensors are torch CUDA tensors (complex128 blocks
[K, p, n_max], float64 grids [N, N, N]) passed by pointer on the current stream.
There is no fallback: a missing library raises ImportError.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB

__all__ = [
    "EacgModel", "EacgParams", "EacgStepInfo", "EacgResult", "EacgError", "lib", "model_from_config",
    "eacg_default_params", "eacg_bytes_required", "eacg_create_system", "eacg_destroy", "eacg_last_error",
    "eacg_get_dims", "eacg_get_plans", "eacg_graph_launches", "eacg_gemm_tile", "eacg_force_gemm_tile", "eacg_get_basis", "eacg_set_psi", "eacg_get_psi", "eacg_density", "eacg_get_potential",
    "eacg_apply_H", "eacg_energy", "eacg_ea_gradient", "eacg_retract", "eacg_step", "eacg_solve",
    "eacg_solve_host", "eacg_profile_enable", "eacg_profile_read", "eacg_launch_count", "EacgKernelStat",
    "eacg_stream_create", "eacg_stream_destroy", "eacg_step_many", "eacg_batching", "eacg_batch_counts", "eacg_overlap_noalloc", "eacg_overlap_c64", "eacg_backproject_c64", "eacg_scf_guess", "System", "STATUS", "EACG_MAX_BANDS", "EACG_MAX_BANDS_DENSE",
]

# band limits of include/eacg.h: transforms / H / density / energy, and the p x p dense calls
EACG_MAX_BANDS = 1024
EACG_MAX_BANDS_DENSE = 512

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EBREAKDOWN", 5: "ENONCOERCIVE",
          6: "ELINESEARCH", 7: "ENAN", 8: "ENOTCONV", 9: "EUNSUPPORTED"}

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class EacgModel(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("natoms", ctypes.c_int), ("pos", _dp), ("Z", _ip), ("rc", _dp),
                ("nproj_per_atom", ctypes.c_int), ("proj_width", ctypes.c_double), ("D", _dp),
                ("ecut", ctypes.c_double), ("N", ctypes.c_int), ("nbands", ctypes.c_int), ("nk", ctypes.c_int),
                ("kfrac", _dp), ("kweight", _dp), ("hartree", ctypes.c_int), ("xc", ctypes.c_int),
                ("occ", ctypes.c_double)]


class EacgParams(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("res_tol", ctypes.c_double), ("fom_rtol", ctypes.c_double),
                ("delta", ctypes.c_double), ("sigma", ctypes.c_double), ("gamma", ctypes.c_double),
                ("eps", ctypes.c_double), ("warm_res", ctypes.c_double), ("switch_res", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("max_warm", ctypes.c_int), ("max_fom", ctypes.c_int),
                ("max_ls", ctypes.c_int), ("precision", ctypes.c_int), ("graphs", ctypes.c_int),
                ("fft_plan", ctypes.c_int), ("method", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("df_transforms", ctypes.c_int)]


class EacgStepInfo(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("rnorm", ctypes.c_double), ("tau", ctypes.c_double),
                ("beta", ctypes.c_double), ("fom_iters_max", ctypes.c_int), ("ls_trials", ctypes.c_int),
                ("phase", ctypes.c_int), ("precision", ctypes.c_int), ("converged", ctypes.c_int),
                ("h_band_apps", ctypes.c_longlong)]


class EacgResult(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("rnorm", ctypes.c_double), ("iterations", ctypes.c_int),
                ("warm_iterations", ctypes.c_int), ("status", ctypes.c_int), ("ls_trials", ctypes.c_int),
                ("h_band_apps", ctypes.c_longlong)]


class EacgKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double), ("units", ctypes.c_double)]


class EacgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB):
        raise ImportError(f"libeacg.so is not built ({LIB}); run paper_2503_16225_gb300.build.build()")
    L = ctypes.CDLL(LIB)
    vp, sp = ctypes.c_void_p, ctypes.c_size_t
    sig = {
        "eacg_default_params": (None, [ctypes.POINTER(EacgParams)]),
        "eacg_bytes_required": (sp, [ctypes.POINTER(EacgModel), ctypes.POINTER(EacgParams), ctypes.POINTER(sp)]),
        "eacg_create_system": (ctypes.c_int, [ctypes.POINTER(EacgModel), ctypes.POINTER(EacgParams), vp,
                                              ctypes.POINTER(vp)]),
        "eacg_destroy": (None, [vp]),
        "eacg_last_error": (ctypes.c_char_p, [vp]),
        "eacg_get_dims": (ctypes.c_int, [vp, _ip, _ip, _ip]),
        "eacg_get_plans": (ctypes.c_int, [vp, _ip, _ip]),
        "eacg_graph_launches": (ctypes.c_longlong, [vp]),
        "eacg_gemm_tile": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "eacg_force_gemm_tile": (ctypes.c_int, [ctypes.c_int]),
        "eacg_get_basis": (ctypes.c_int, [vp, vp]),
        "eacg_set_psi": (ctypes.c_int, [vp, vp]),
        "eacg_get_psi": (ctypes.c_int, [vp, vp]),
        "eacg_density": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
        "eacg_get_potential": (ctypes.c_int, [vp, vp]),
        "eacg_apply_H": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
        "eacg_energy": (ctypes.c_int, [vp, vp, _dp, vp, vp, _dp, ctypes.c_int]),
        "eacg_ea_gradient": (ctypes.c_int, [vp, vp, vp, _ip, ctypes.c_int]),
        "eacg_retract": (ctypes.c_int, [vp, vp, vp, ctypes.c_double, vp, vp]),
        "eacg_step": (ctypes.c_int, [vp, ctypes.POINTER(EacgStepInfo)]),
        "eacg_step_many": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(EacgStepInfo), _ip,
                                          ctypes.c_int]),
        "eacg_batching": (ctypes.c_int, [ctypes.c_int]),
        "eacg_batch_counts": (ctypes.c_int, [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
        "eacg_solve": (ctypes.c_int, [vp, ctypes.POINTER(EacgResult)]),
        "eacg_solve_host": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(EacgResult)]),
        "eacg_profile_enable": (ctypes.c_int, [vp, ctypes.c_int]),
        "eacg_profile_read": (ctypes.c_int, [vp, ctypes.POINTER(EacgKernelStat), ctypes.c_int]),
        "eacg_launch_count": (ctypes.c_longlong, []),
        "eacg_stream_create": (ctypes.c_int, [ctypes.POINTER(vp)]),
        "eacg_stream_destroy": (ctypes.c_int, [vp]),
        "eacg_overlap_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]),
        "eacg_overlap_c64": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp,
                                            ctypes.c_int, vp]),
        "eacg_backproject_c64": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                                                vp, ctypes.c_int, vp]),
        "eacg_scf_guess": (ctypes.c_int, [vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                          _ip, _dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(sys, code):
    if code != 0:
        msg = lib.eacg_last_error(sys).decode() if sys else ""
        raise EacgError(code, msg)


class _ModelBuffers:
    """Keeps the host arrays of an EacgModel alive."""

    def __init__(self, cfg):
        import numpy as np
        self.pos = np.ascontiguousarray(cfg["pos"], np.float64).reshape(-1)
        self.Z = np.ascontiguousarray(cfg["Z"], np.int32).reshape(-1)
        self.rc = np.ascontiguousarray(cfg["rc"], np.float64).reshape(-1)
        self.D = np.ascontiguousarray(cfg["D"], np.float64).reshape(-1)
        self.kfrac = np.ascontiguousarray(cfg["kfrac"], np.float64).reshape(-1)
        self.kw = np.ascontiguousarray(cfg["kweight"], np.float64).reshape(-1)
        if self.pos.size == 0:
            self.pos = np.zeros(3)
            self.Z = np.zeros(1, np.int32)
            self.rc = np.ones(1)
            self.D = np.zeros(2)
        self.m = EacgModel(
            a=float(cfg["a"]), natoms=int(len(cfg["Z"])), pos=self.pos.ctypes.data_as(_dp),
            Z=self.Z.ctypes.data_as(_ip), rc=self.rc.ctypes.data_as(_dp),
            nproj_per_atom=int(cfg["nproj_per_atom"]), proj_width=float(cfg["proj_width"]),
            D=self.D.ctypes.data_as(_dp), ecut=float(cfg["ecut"]), N=int(cfg["N"]), nbands=int(cfg["nbands"]),
            nk=int(len(self.kw)), kfrac=self.kfrac.ctypes.data_as(_dp), kweight=self.kw.ctypes.data_as(_dp),
            hartree=int(cfg["hartree"]), xc=int(cfg["xc"]), occ=float(cfg["occ"]))


def model_from_config(cfg):
    return _ModelBuffers(cfg)


# ----------------------------------------------------------------------------- C names
def eacg_default_params(**overrides) -> EacgParams:
    p = EacgParams()
    lib.eacg_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def eacg_bytes_required(cfg, params=None):
    mb = model_from_config(cfg)
    per = ctypes.c_size_t(0)
    n = lib.eacg_bytes_required(ctypes.byref(mb.m), ctypes.byref(params) if params else None, ctypes.byref(per))
    return int(n), int(per.value)


def eacg_create_system(cfg, params=None, stream=None):
    mb = model_from_config(cfg)
    h = ctypes.c_void_p()
    code = lib.eacg_create_system(ctypes.byref(mb.m), ctypes.byref(params) if params else None, _stream(stream),
                                  ctypes.byref(h))
    if code != 0:
        raise EacgError(code, "eacg_create_system failed")
    return h


def eacg_destroy(sys):
    lib.eacg_destroy(sys)


def eacg_last_error(sys):
    return lib.eacg_last_error(sys).decode()


def eacg_get_dims(sys, K):
    nk = (ctypes.c_int * K)()
    n_max, ncols = ctypes.c_int(), ctypes.c_int()
    _check(sys, lib.eacg_get_dims(sys, nk, ctypes.byref(n_max), ctypes.byref(ncols)))
    return list(nk), n_max.value, ncols.value


def eacg_get_basis(sys, m_dev):
    _check(sys, lib.eacg_get_basis(sys, _ptr(m_dev)))


def eacg_set_psi(sys, psi):
    _check(sys, lib.eacg_set_psi(sys, _ptr(psi)))


def eacg_get_plans(sys):
    """(plan of the FP64 transforms, plan of the FP32 transforms)."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(sys, lib.eacg_get_plans(sys, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def eacg_graph_launches(sys):
    return int(lib.eacg_graph_launches(sys))


def eacg_gemm_tile(m, n, L, precision):
    return int(lib.eacg_gemm_tile(m, n, L, precision))


def eacg_force_gemm_tile(groups):
    _check(None, lib.eacg_force_gemm_tile(groups))


def eacg_get_psi(sys, out):
    _check(sys, lib.eacg_get_psi(sys, _ptr(out)))


def eacg_density(sys, psi, rho=None, precision=0):
    _check(sys, lib.eacg_density(sys, _ptr(psi), _ptr(rho), precision))


def eacg_get_potential(sys, out):
    _check(sys, lib.eacg_get_potential(sys, _ptr(out)))


def eacg_apply_H(sys, psi, hpsi, precision=0):
    _check(sys, lib.eacg_apply_H(sys, _ptr(psi), _ptr(hpsi), precision))


def eacg_energy(sys, psi, lam=None, res=None, precision=0):
    terms = (ctypes.c_double * 6)()
    rn = ctypes.c_double()
    _check(sys, lib.eacg_energy(sys, _ptr(psi), terms, _ptr(lam), _ptr(res), ctypes.byref(rn), precision))
    return list(terms), rn.value


def eacg_ea_gradient(sys, psi, g, K, precision=0):
    it = (ctypes.c_int * K)()
    _check(sys, lib.eacg_ea_gradient(sys, _ptr(psi), _ptr(g), it, precision))
    return list(it)


def eacg_retract(sys, phi, eta, tau, phi_out, teta_out=None):
    _check(sys, lib.eacg_retract(sys, _ptr(phi), _ptr(eta), float(tau), _ptr(phi_out), _ptr(teta_out)))


def eacg_step(sys):
    info = EacgStepInfo()
    code = lib.eacg_step(sys, ctypes.byref(info))
    _check(sys, code)
    return info


def eacg_step_many(systems, window_us=200, check=True):
    """One step of each system (handles), taken together with batched transform launches;
    returns (step infos, per-system status codes)."""
    n = len(systems)
    arr = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in systems])
    infos = (EacgStepInfo * n)()
    sts = (ctypes.c_int * n)()
    code = lib.eacg_step_many(arr, n, infos, sts, int(window_us))
    if check and code != 0:
        bad = next(i for i in range(n) if sts[i] != 0) if any(sts[i] for i in range(n)) else 0
        _check(systems[bad], code)
    return list(infos), list(sts)


def eacg_batching(window_us):
    """Process-wide batching of concurrent eacg_step calls (window_us >= 0), or off (-1)."""
    _check(None, lib.eacg_batching(int(window_us)))


def eacg_batch_counts():
    """(batched transform groups, system requests covered) since the process started."""
    g, m = ctypes.c_longlong(), ctypes.c_longlong()
    _check(None, lib.eacg_batch_counts(ctypes.byref(g), ctypes.byref(m)))
    return g.value, m.value


def eacg_solve(sys, check=True):
    res = EacgResult()
    code = lib.eacg_solve(sys, ctypes.byref(res))
    if check:
        _check(sys, code)
    return res


def eacg_solve_host(sys, psi0_host, psi_out_host, check=True):
    res = EacgResult()
    code = lib.eacg_solve_host(sys, ctypes.c_void_p(psi0_host.data_ptr()),
                               ctypes.c_void_p(psi_out_host.data_ptr()), ctypes.byref(res))
    if check:
        _check(sys, code)
    return res


def eacg_profile_enable(sys, on=1):
    _check(sys, lib.eacg_profile_enable(sys, int(on)))


def eacg_profile_read(sys):
    """{kernel name: {launches, ms, bytes, units}} since eacg_profile_enable (then cleared)."""
    buf = (EacgKernelStat * 32)()
    n = lib.eacg_profile_read(sys, buf, 32)
    if n < 0:
        raise EacgError(-n, eacg_last_error(sys))
    return {buf[i].name.decode(): {"launches": buf[i].launches, "ms": buf[i].ms, "bytes": buf[i].bytes,
                                   "flops": buf[i].flops, "units": buf[i].units} for i in range(n)}


def eacg_launch_count():
    return int(lib.eacg_launch_count())


def eacg_stream_create():
    """Handle (int) of a new non-blocking CUDA stream owned by the caller."""
    h = ctypes.c_void_p()
    _check(None, lib.eacg_stream_create(ctypes.byref(h)))
    return int(h.value)


def eacg_stream_destroy(stream):
    _check(None, lib.eacg_stream_destroy(ctypes.c_void_p(stream)))


def eacg_overlap_noalloc(a, b, c, stream=None):
    """c[k] = a[k]^* b[k] for complex128 tensors a, b [K, p, n] and c [K, p, p] (column-major
    p x p per k), through the allocation-free entry point; returns the eacg_status code."""
    import torch
    K, p, n = a.shape
    for t, shape in ((a, (K, p, n)), (b, (K, p, n)), (c, (K, p, p))):
        if (tuple(t.shape) != shape or t.dtype != torch.complex128 or not t.is_cuda
                or not t.is_contiguous()):
            raise ValueError(f"eacg_overlap_noalloc: expected contiguous complex128 CUDA tensors "
                             f"a, b [K, p, n] and c [K, p, p]; got {tuple(t.shape)} {t.dtype}")
    return int(lib.eacg_overlap_noalloc(K, n, p, _ptr(a), _ptr(b), _ptr(c), _stream(stream)))


def eacg_scf_guess(sys, psi0, tol=0.1, alpha=0.5, max_scf=100, eig_tol=1e-10):
    """SCF initial guess (Sec. 5.2) from the device block psi0 [K, p, n_max]; returns the
    density differences ||rho_out - rho_in||_2 of the steps taken (the last is below tol)."""
    steps = ctypes.c_int(0)
    hist = (ctypes.c_double * max_scf)()
    _check(sys, lib.eacg_scf_guess(sys, _ptr(psi0), float(tol), float(alpha), int(max_scf), float(eig_tol),
                                   ctypes.byref(steps), hist))
    return list(hist[:steps.value])


def eacg_backproject_c64(a, q, c, method=1, stream=None):
    """c[k] += a[k] q[k] for complex64 a [K, m, L], complex128 q [K, n, m] and complex128 c
    [K, n, L] (column-major per k); method 1 = tensor cores, 0 = SIMT FP32.  Returns the status."""
    K, m, L = a.shape
    n = q.shape[1]
    return int(lib.eacg_backproject_c64(K, L, m, n, _ptr(a), _ptr(q), _ptr(c), int(method), _stream(stream)))


def eacg_overlap_c64(a, b, c, method=1, stream=None):
    """c[k] = a[k]^* b[k] for complex64 tensors a [K, m, L], b [K, n, L] and complex128 c [K, n, m]
    (column-major m x n per k); method 1 = tensor cores (3 x TF32), 0 = SIMT FP32.  Returns the
    eacg_status code."""
    K, m, L = a.shape
    n = b.shape[1]
    return int(lib.eacg_overlap_c64(K, L, m, n, _ptr(a), _ptr(b), _ptr(c), int(method), _stream(stream)))


class System:
    """Owning wrapper: one Kohn-Sham problem resident on the current CUDA device."""

    def __init__(self, cfg, params=None, stream=None):
        import torch
        self.cfg = cfg
        self.params = params or eacg_default_params()
        self.h = eacg_create_system(cfg, self.params, stream)
        self.K = len(cfg["kweight"])
        self.p = int(cfg["nbands"])
        self.N = int(cfg["N"])
        self.nk, self.n_max, self.ncols = eacg_get_dims(self.h, self.K)
        self.torch = torch

    def close(self):
        if self.h:
            eacg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def block(self):
        return self.torch.zeros((self.K, self.p, self.n_max), dtype=self.torch.complex128, device="cuda")

    def grid(self):
        return self.torch.zeros((self.N,) * 3, dtype=self.torch.float64, device="cuda")

    def basis(self):
        m = self.torch.zeros((self.K, self.n_max, 3), dtype=self.torch.int32, device="cuda")
        eacg_get_basis(self.h, m)
        return m
