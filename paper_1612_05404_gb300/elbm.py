"""Thin ctypes binding of the C ABI in include/elbm.h (libelbm.so).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels. There is no CPU fallback; if the library cannot be loaded the
import of this module's functions raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libelbm.so")

OK, W_POISSON_NOCONV, E_INVAL, E_NOMEM, E_CUDA, E_NUMERIC, E_STATE = 0, 1, -1, -2, -3, -4, -5
F_RHO, F_U, F_PHI, F_Q, F_ALPHA, F_NU, F_POP, F_GPOP, F_DIAG = (1 << i for i in range(9))
NDIAG = 24
DIAG_NAMES = [
    "mass", "mom_x", "mom_y", "mom_z", "charge", "alpha_min", "alpha_max", "alpha_mean",
    "n_shortcut", "n_noroot", "n_clipped", "poisson_sweeps", "poisson_resid", "max_h_error",
    "max_u", "n_nonfinite", "q_mean", "step", "poisson_sweeps_total", "n_guarded",
    "n_guard_failed", "n_learned_fallback", "inlet_scale", "flags_undiagnosed",
]
EXPORTS = ["elbm_init", "elbm_step", "elbm_fields", "elbm_fields_size", "elbm_free",
           "elbm_strerror", "elbm_velocity_set", "elbm_velocity_set_of", "elbm_pass_times", "elbm_density_noalloc",
           "elbm_alpha_eval", "elbm_alpha_features", "elbm_alpha_harvest", "elbm_mlp_forward",
           "elbm_mlp_workspace_floats", "elbm_mlp_grad", "elbm_mlp_adam", "elbm_mlp_train",
           "elbm_batch_create"]
MLP_NIN = 20
MLP_NPARAM = 5569
NOALLOC_MAX_SITES = 16384 * 1024

_FACE = {"periodic": 0, "wall": 1}
_PHI = {"periodic": 0, "dirichlet": 1, "neumann": 2}
_CHARGE = {"none": 0, "conserved": 1, "xi": 2, "transport": 3}
_FEL = {"qe": 0, "full": 1}
_ALPHA = {"entropic": 0, "bgk": 1, "learned": 2}
_PREC = {"fp64": 0, "fp32": 1, "bf16": 2}
_APREC = {"fp64": 0, "fp32": 1, "fp32_fast": 2}


class ElbmError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("face_bc", ctypes.c_int * 6), ("phi_bc", ctypes.c_int * 6),
        ("phi_axis", ctypes.c_int), ("charge_model", ctypes.c_int), ("force_el", ctypes.c_int),
        ("neutralize", ctypes.c_int), ("poisson_solver", ctypes.c_int), ("poisson_maxit", ctypes.c_int),
        ("poisson_fixed_sweeps", ctypes.c_int), ("poisson_check_every", ctypes.c_int),
        ("alpha_mode", ctypes.c_int), ("precision", ctypes.c_int),
        ("alpha_precision", ctypes.c_int), ("store_macro", ctypes.c_int),
        ("diag_every", ctypes.c_int), ("profile", ctypes.c_int), ("graph", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("phi_lo", ctypes.c_double), ("phi_hi", ctypes.c_double), ("phi_solid", ctypes.c_double),
        ("nu0", ctypes.c_double), ("nu_inf", ctypes.c_double), ("lam", ctypes.c_double),
        ("n_carreau", ctypes.c_double),
        ("G", ctypes.c_double), ("Gw", ctypes.c_double), ("rho0", ctypes.c_double),
        ("eps_kappa", ctypes.c_double), ("sigma_liq", ctypes.c_double),
        ("sigma_gas", ctypes.c_double), ("Dq", ctypes.c_double), ("E_ext", ctypes.c_double * 3),
        ("Q_b", ctypes.c_double), ("Q_s", ctypes.c_double), ("K_d", ctypes.c_double),
        ("xi_b", ctypes.c_double), ("xi_s", ctypes.c_double), ("theta_width", ctypes.c_double),
        ("sor_omega", ctypes.c_double), ("poisson_tol", ctypes.c_double),
        ("alpha_eq_tol", ctypes.c_double), ("rho_in", ctypes.c_double), ("rho_out", ctypes.c_double),
        ("cuda_stream", ctypes.c_void_p),
        ("mlp", ctypes.c_void_p),
        ("eps_face", ctypes.c_int), ("carreau_lagged", ctypes.c_int),
        ("alpha_h_tol", ctypes.c_double),
        ("velset", ctypes.c_int),
    ]


class InitFields(ctypes.Structure):
    _fields_ = [("mask", ctypes.POINTER(ctypes.c_ubyte)),
                ("rho0", ctypes.POINTER(ctypes.c_double)), ("u0", ctypes.POINTER(ctypes.c_double)),
                ("q0", ctypes.POINTER(ctypes.c_double)), ("u_in", ctypes.POINTER(ctypes.c_double)),
                ("f0", ctypes.POINTER(ctypes.c_double)),
                ("inlet_region", ctypes.POINTER(ctypes.c_ubyte))]


_lib = None


def lib():
    """Load libelbm.so (built by paper_1612_05404_gb300.build). Raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libelbm.so not built ({LIB_PATH}); run paper_1612_05404_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.elbm_init.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(InitFields), ctypes.c_int,
                                ctypes.POINTER(vp)]
        L.elbm_init.restype = ctypes.c_int
        L.elbm_step.argtypes = [vp, ctypes.c_int]
        L.elbm_step.restype = ctypes.c_int
        L.elbm_fields.argtypes = [vp, ctypes.c_uint, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t]
        L.elbm_fields.restype = ctypes.c_int
        L.elbm_fields_size.argtypes = [vp, ctypes.c_uint]
        L.elbm_fields_size.restype = ctypes.c_size_t
        L.elbm_free.argtypes = [vp]
        L.elbm_free.restype = None
        L.elbm_strerror.argtypes = [ctypes.c_int]
        L.elbm_strerror.restype = ctypes.c_char_p
        L.elbm_velocity_set.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        L.elbm_velocity_set.restype = ctypes.c_int
        L.elbm_velocity_set_of.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        L.elbm_velocity_set_of.restype = ctypes.c_int
        L.elbm_pass_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.elbm_pass_times.restype = ctypes.c_int
        L.elbm_density_noalloc.argtypes = [vp, vp, ctypes.c_longlong, vp, vp, vp]
        L.elbm_density_noalloc.restype = ctypes.c_int
        L.elbm_alpha_eval.argtypes = [vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_double, vp, vp, vp, vp, vp, vp]
        L.elbm_alpha_eval.restype = ctypes.c_int
        L.elbm_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.elbm_batch_create.restype = ctypes.c_int
        ll, f = ctypes.c_longlong, ctypes.c_float
        L.elbm_alpha_features.argtypes = [vp, ll, vp, vp, vp]
        L.elbm_alpha_harvest.argtypes = [vp, ll, ctypes.c_double, vp, vp, vp, vp]
        L.elbm_mlp_forward.argtypes = [vp, ll, vp, ctypes.c_int, vp, vp]
        L.elbm_mlp_workspace_floats.argtypes = [ll]
        L.elbm_mlp_workspace_floats.restype = ll
        L.elbm_mlp_grad.argtypes = [vp, vp, ll, vp, vp, vp, vp, vp]
        L.elbm_mlp_adam.argtypes = [vp, vp, vp, vp, ctypes.c_int, f, f, f, f, vp]
        L.elbm_mlp_train.argtypes = [vp, vp, ll, vp, vp, vp, ctypes.c_int, ctypes.c_int, ll, f,
                                     ctypes.c_ulonglong, vp, vp, vp]
        for name in ("elbm_alpha_features", "elbm_alpha_harvest", "elbm_mlp_forward", "elbm_mlp_grad",
                     "elbm_mlp_adam", "elbm_mlp_train"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().elbm_strerror(int(code)).decode()


VSET = {3: 0, 2: 1}  # lattice dimension -> ELBM_VSET_D3Q19 / ELBM_VSET_D2Q9


def velocity_set(dim: int = 3):
    """(c (Q, 3), w (Q,)) of the D3Q19 set (dim 3) or the D2Q9 set (dim 2)."""
    c = (ctypes.c_int * 57)()
    w = (ctypes.c_double * 19)()
    Q = lib().elbm_velocity_set_of(VSET[dim], c, w)
    if Q < 0:
        raise ElbmError(Q, "elbm_velocity_set_of")
    return np.array(list(c)[:3 * Q]).reshape(Q, 3), np.array(list(w)[:Q])


def make_params(cfg: dict, stream=None) -> Params:
    P = Params()
    P.nx, P.ny, P.nz = cfg["shape"]
    for i, v in enumerate(cfg["face_bc"]):
        P.face_bc[i] = _FACE[v]
    for i, v in enumerate(cfg["phi_bc"]):
        P.phi_bc[i] = _PHI[v]
    P.phi_axis = cfg["phi_axis"]
    P.charge_model = _CHARGE[cfg["charge_model"]]
    P.force_el = _FEL[cfg["force_el"]]
    P.neutralize = int(cfg["neutralize"])
    P.poisson_solver = {"sor": 0, "mg": 1}[cfg.get("poisson_solver", "sor")]
    P.poisson_maxit = cfg["poisson_maxit"] if P.poisson_solver == 0 else cfg.get("poisson_mg_cycles", 50)
    P.poisson_fixed_sweeps = cfg["poisson_fixed_sweeps"]
    P.poisson_check_every = cfg.get("poisson_check_every", 8)
    P.alpha_mode = _ALPHA[cfg["alpha_mode"]]
    P.precision = _PREC[cfg["precision"]]
    P.alpha_precision = _APREC[cfg.get("alpha_precision", "fp64")]
    P.store_macro = int(cfg.get("store_macro", 1))
    P.diag_every = int(cfg.get("diag_every", 1))
    P.profile = int(cfg.get("profile", 0))
    P.graph = int(cfg.get("graph", 1))
    P.autotune = int(cfg.get("autotune", 0))
    P.phi_lo, P.phi_hi, P.phi_solid = cfg["phi_lo"], cfg["phi_hi"], cfg["phi_solid"]
    P.nu0, P.nu_inf, P.lam, P.n_carreau = cfg["nu0"], cfg["nu_inf"], cfg["lambda"], cfg["n_carreau"]
    P.G, P.Gw, P.rho0 = cfg["G"], cfg["Gw"], cfg["rho0"]
    P.eps_kappa = cfg["eps_kappa"]
    P.sigma_liq, P.sigma_gas, P.Dq = cfg["sigma_liq"], cfg["sigma_gas"], cfg["Dq"]
    for i in range(3):
        P.E_ext[i] = cfg["E_ext"][i]
    P.Q_b, P.Q_s, P.K_d = cfg["Q_b"], cfg["Q_s"], cfg["K_d"]
    P.xi_b, P.xi_s, P.theta_width = cfg["xi_b"], cfg["xi_s"], cfg["theta_width"]
    P.sor_omega, P.poisson_tol = cfg["sor_omega"], cfg["poisson_tol"]
    P.alpha_eq_tol = cfg["alpha_eq_tol"]
    P.rho_in, P.rho_out = cfg["rho_in"], cfg["rho_out"]
    P.cuda_stream = stream
    P.eps_face = {"arithmetic": 0, "harmonic": 1}[cfg.get("eps_face", "arithmetic")]
    P.carreau_lagged = int(cfg.get("carreau_lagged", 0))
    P.alpha_h_tol = float(cfg.get("alpha_h_tol", 0.0))
    P.velset = VSET[int(cfg.get("dim", 3))]
    mlp = cfg.get("mlp")
    P.mlp = None if mlp is None else mlp.data_ptr()
    return P


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _cur_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def density_noalloc(f_ptr: int, mask_ptr, n_sites: int, rho_ptr: int, mass_ptr: int, stream=None) -> int:
    """elbm_density_noalloc on caller-owned device pointers; returns the status."""
    return lib().elbm_density_noalloc(ctypes.c_void_p(f_ptr), ctypes.c_void_p(mask_ptr or 0),
                                      int(n_sites), ctypes.c_void_p(rho_ptr), ctypes.c_void_p(mass_ptr),
                                      stream)


def alpha_eval(d, aprec="fp32", eq_tol=1e-5, mlp=None, with_delta=False, stream=None):
    """elbm_alpha_eval on a CUDA tensor of FP32 deviations d (19, n).

    Returns (alpha FP64 [n], herr FP32 [n], status int32 [n], delta FP32
    (19, n) or None) as CUDA tensors, computed on `stream` (default: the
    current torch stream)."""
    import torch
    if not (d.is_cuda and d.dtype == torch.float32 and d.dim() == 2 and d.shape[0] == 19):
        raise ValueError("d must be a CUDA float32 tensor of shape (19, n)")
    d = d.contiguous()
    n = d.shape[1]
    alpha = torch.empty(n, dtype=torch.float64, device=d.device)
    herr = torch.empty(n, dtype=torch.float32, device=d.device)
    status = torch.empty(n, dtype=torch.int32, device=d.device)
    delta = torch.empty((19, n), dtype=torch.float32, device=d.device) if with_delta else None
    rc = lib().elbm_alpha_eval(ctypes.c_void_p(d.data_ptr()), n, _APREC[aprec], float(eq_tol),
                               ctypes.c_void_p(0 if mlp is None else mlp.data_ptr()),
                               ctypes.c_void_p(alpha.data_ptr()), ctypes.c_void_p(herr.data_ptr()),
                               ctypes.c_void_p(status.data_ptr()),
                               ctypes.c_void_p(0 if delta is None else delta.data_ptr()),
                               stream if stream is not None else _cur_stream())
    if rc != 0:
        raise ElbmError(rc)
    return alpha, herr, status, delta


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _check(rc, what):
    if rc != 0:
        raise ElbmError(rc, what)


def _cuda_f32(t, shape0=None):
    import torch
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA float32 tensor")
    if shape0 is not None and t.shape[0] != shape0:
        raise ValueError(f"expected leading dimension {shape0}")
    return t


def alpha_features(d, stream=None):
    """Features X (20, n) and S (n) of sites given as FP32 deviations (19, n)."""
    import torch
    _cuda_f32(d, 19)
    n = d.shape[1]
    X = torch.empty((MLP_NIN, n), dtype=torch.float32, device=d.device)
    S = torch.empty(n, dtype=torch.float32, device=d.device)
    _check(lib().elbm_alpha_features(_p(d), n, _p(X), _p(S), stream or _cur_stream()), "elbm_alpha_features")
    return X, S


def alpha_harvest(d, eq_tol=1e-5, stream=None):
    """Training pairs (X (20, n), y (n), keep (n) int32) of FP32 deviation sites."""
    import torch
    _cuda_f32(d, 19)
    n = d.shape[1]
    X = torch.empty((MLP_NIN, n), dtype=torch.float32, device=d.device)
    y = torch.empty(n, dtype=torch.float32, device=d.device)
    keep = torch.empty(n, dtype=torch.int32, device=d.device)
    _check(lib().elbm_alpha_harvest(_p(d), n, float(eq_tol), _p(X), _p(y), _p(keep), stream or _cur_stream()),
           "elbm_alpha_harvest")
    return X, y, keep


def mlp_forward(X, theta, arith="bf16_tc", stream=None):
    import torch
    _cuda_f32(X, MLP_NIN)
    _cuda_f32(theta)
    o = torch.empty(X.shape[1], dtype=torch.float32, device=X.device)
    _check(lib().elbm_mlp_forward(_p(X), X.shape[1], _p(theta), {"fp32": 0, "bf16_tc": 1}[arith], _p(o),
                                  stream or _cur_stream()), "elbm_mlp_forward")
    return o


def mlp_grad(X, y, theta, stream=None):
    """(grad (NPARAM,), loss (1,)) of the mean squared error over all samples."""
    import torch
    n = X.shape[1]
    g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=X.device)
    L = torch.empty(1, dtype=torch.float32, device=X.device)
    work = torch.empty(int(lib().elbm_mlp_workspace_floats(n)), dtype=torch.float32, device=X.device)
    _check(lib().elbm_mlp_grad(_p(_cuda_f32(X, MLP_NIN)), _p(_cuda_f32(y)), n, _p(_cuda_f32(theta)), _p(g), _p(L),
                               _p(work), stream or _cur_stream()), "elbm_mlp_grad")
    return g, L


def mlp_adam(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().elbm_mlp_adam(_p(theta), _p(g), _p(m), _p(v), int(t), float(lr), float(beta1), float(beta2),
                               float(eps), stream or _cur_stream()), "elbm_mlp_adam")


def mlp_train(X, y, theta, m, v, t0, steps, batch, lr, seed, stream=None):
    """`steps` Adam minibatch steps in place on theta, m, v; returns the
    per-step minibatch losses (CUDA tensor)."""
    import torch
    n = X.shape[1]
    hist = torch.empty(max(steps, 1), dtype=torch.float32, device=X.device)
    work = torch.empty(int(lib().elbm_mlp_workspace_floats(batch)) + MLP_NPARAM, dtype=torch.float32,
                       device=X.device)
    _check(lib().elbm_mlp_train(_p(_cuda_f32(X, MLP_NIN)), _p(_cuda_f32(y)), n, _p(theta), _p(m), _p(v), int(t0),
                                int(steps), int(batch), float(lr), int(seed), _p(hist), _p(work),
                                stream or _cur_stream()), "elbm_mlp_train")
    return hist[:steps]


class Sim:
    """One lattice on the GPU driven through the C ABI."""

    def __init__(self, cfg: dict, fields: dict, stream=None):
        self.cfg = cfg
        nx, ny, nz = cfg["shape"]
        self.N = nx * ny * nz
        self._keep = {}
        for k in ("rho", "u", "q", "u_in", "f"):
            if k in fields and fields[k] is not None:
                self._keep[k] = np.ascontiguousarray(fields[k], dtype=np.float64).reshape(-1)
        for k in ("mask", "inlet_region"):
            a = fields.get(k)
            self._keep[k] = None if a is None else np.ascontiguousarray(a, dtype=np.uint8).reshape(-1)
        IF = InitFields()
        m = self._keep["mask"]
        IF.mask = None if m is None else m.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        r = self._keep["inlet_region"]
        IF.inlet_region = None if r is None else r.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        IF.rho0 = _dptr(self._keep.get("rho"))
        IF.u0 = _dptr(self._keep.get("u"))
        IF.q0 = _dptr(self._keep.get("q"))
        IF.u_in = _dptr(self._keep.get("u_in"))
        IF.f0 = _dptr(self._keep.get("f"))
        self.P = make_params(cfg, stream if stream is not None else _cur_stream())
        h = ctypes.c_void_p()
        rc = lib().elbm_init(ctypes.byref(self.P), ctypes.byref(IF), 1, ctypes.byref(h))
        if rc != OK:
            raise ElbmError(rc, "elbm_init")
        self.h = h
        self.last_status = OK
        self._keep = None  # elbm_init has copied the host fields

    def step(self, n: int = 1) -> int:
        rc = lib().elbm_step(self.h, int(n))
        if rc < 0:
            raise ElbmError(rc, "elbm_step")
        self.last_status = rc
        return rc

    def fields(self, mask: int, out=None) -> np.ndarray:
        n = lib().elbm_fields_size(self.h, mask)
        if out is None:
            out = np.empty(n, dtype=np.float64)
        rc = lib().elbm_fields(self.h, mask, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size)
        if rc != OK:
            raise ElbmError(rc, "elbm_fields")
        return out

    def get(self, name: str) -> np.ndarray:
        sel = {"rho": F_RHO, "u": F_U, "phi": F_PHI, "q": F_Q, "alpha": F_ALPHA, "nu": F_NU,
               "f": F_POP, "g": F_GPOP, "diag": F_DIAG}[name]
        return self.fields(sel)

    def pass_times(self) -> dict:
        out = (ctypes.c_double * 8)()
        rc = lib().elbm_pass_times(self.h, out, 8)
        if rc != OK:
            raise ElbmError(rc, "elbm_pass_times")
        keys = ["moments_ms", "poisson_ms", "collide_ms", "reduce_ms", "steps", "collide_launches",
                "sweeps", "launches"]
        return dict(zip(keys, list(out)))

    def diag(self) -> dict:
        return dict(zip(DIAG_NAMES, self.fields(F_DIAG).tolist()))

    def close(self):
        if getattr(self, "h", None):
            lib().elbm_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Lattices advanced together, one CUDA graph launch per step
    (elbm_batch_create). The batch keeps references to its Sim instances; step
    them only through the batch; read fields from each instance."""

    def __init__(self, sims, pipeline=False, span=1, stream=None):
        self.sims = list(sims)
        arr = (ctypes.c_void_p * len(self.sims))(*[s.h.value for s in self.sims])
        h = ctypes.c_void_p()
        flags = (1 if pipeline else 0) | (int(span) << 8 if span > 1 else 0)  # ELBM_BATCH_PIPELINE, _SPAN(k)
        rc = lib().elbm_batch_create(arr, len(self.sims), flags,
                                     stream if stream is not None else _cur_stream(), ctypes.byref(h))
        if rc != OK:
            raise ElbmError(rc, "elbm_batch_create")
        self.h = h

    def step(self, n: int = 1) -> int:
        rc = lib().elbm_step(self.h, int(n))
        if rc < 0:
            raise ElbmError(rc, "elbm_step (batch)")
        return rc

    def close(self):
        if getattr(self, "h", None):
            lib().elbm_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

