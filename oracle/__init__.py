"""Plain FP64 CPU oracle of the charged entropic lattice Boltzmann step.

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library and
its Python binding never import it, and it imports nothing from them; the one
module both sides read is ``paper_1612_05404_gb300.workloads`` (seeded input
fields and parameter dictionaries, none of the method's arithmetic).

The arithmetic lives in ``elbm_oracle.c`` (plain C, FP64, no fast-math); this
file compiles it with gcc and wraps it with ctypes. Every function cites the
passage of Lauricella et al. (arXiv:1612.05404) it follows in the C source.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "elbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libelbm_oracle.so")
_lock = threading.Lock()
_lib = None

FLUID, SOLID, INLET, OUTLET = 0, 1, 2, 3
NDIAG = 20
DIAG_NAMES = [
    "mass", "mom_x", "mom_y", "mom_z", "charge", "alpha_min", "alpha_max",
    "alpha_mean", "n_shortcut", "n_noroot", "n_clipped", "poisson_sweeps",
    "poisson_resid", "max_h_error", "max_u", "H_total", "q_mean",
    "F_x", "F_y", "F_z",
]

_FACE = {"periodic": 0, "wall": 1}
_PHI = {"periodic": 0, "dirichlet": 1, "neumann": 2}
_CHARGE = {"none": 0, "conserved": 1, "xi": 2, "transport": 3}
_FEL = {"qe": 0, "full": 1}
_ALPHA = {"entropic": 0, "bgk": 1}
_EPS_FACE = {"arithmetic": 0, "harmonic": 1}


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("nz", ctypes.c_int), ("face_bc", ctypes.c_int * 6),
        ("phi_bc", ctypes.c_int * 6), ("phi_axis", ctypes.c_int),
        ("charge_model", ctypes.c_int), ("force_el", ctypes.c_int),
        ("neutralize", ctypes.c_int), ("poisson_maxit", ctypes.c_int),
        ("poisson_fixed_sweeps", ctypes.c_int), ("alpha_mode", ctypes.c_int),
        ("eps_face", ctypes.c_int), ("carreau_lagged", ctypes.c_int), ("pad1", ctypes.c_int),
        ("phi_lo", ctypes.c_double), ("phi_hi", ctypes.c_double),
        ("phi_solid", ctypes.c_double),
        ("nu0", ctypes.c_double), ("nu_inf", ctypes.c_double),
        ("lam", ctypes.c_double), ("n_carreau", ctypes.c_double),
        ("G", ctypes.c_double), ("Gw", ctypes.c_double), ("rho0", ctypes.c_double),
        ("eps_kappa", ctypes.c_double),
        ("sigma_liq", ctypes.c_double), ("sigma_gas", ctypes.c_double),
        ("Dq", ctypes.c_double), ("E_ext", ctypes.c_double * 3),
        ("Q_b", ctypes.c_double), ("Q_s", ctypes.c_double), ("K_d", ctypes.c_double),
        ("xi_b", ctypes.c_double), ("xi_s", ctypes.c_double),
        ("theta_width", ctypes.c_double),
        ("sor_omega", ctypes.c_double), ("poisson_tol", ctypes.c_double),
        ("alpha_eq_tol", ctypes.c_double),
        ("rho_in", ctypes.c_double), ("rho_out", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libelbm_oracle.so (gcc, -O2)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def substituted(path: str):
    """Test infrastructure: inside the block every function of this module
    runs from the library at `path`, another build of elbm_oracle.c (a copy
    with a planted mistake, to show that the pins catch it)."""
    global _lib
    old = lib()
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = old


def _configure(L):
    """Argument and result types of the oracle's C entry points."""
    dp = ctypes.POINTER(ctypes.c_double)
    u8p = ctypes.POINTER(ctypes.c_ubyte)
    pp = ctypes.POINTER(Params)
    L.orc_Q.argtypes = [ctypes.c_int]
    L.orc_lattice.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, dp]
    L.orc_feq.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
    L.orc_H.argtypes = [ctypes.c_int, dp]
    L.orc_H.restype = ctypes.c_double
    L.orc_h.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double]
    L.orc_h.restype = ctypes.c_double
    L.orc_h_prime0.argtypes = [ctypes.c_int, dp, dp]
    L.orc_h_prime0.restype = ctypes.c_double
    L.orc_alpha.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp]
    L.orc_alpha_bisect.argtypes = [ctypes.c_int, dp, dp]
    L.orc_alpha_bisect.restype = ctypes.c_double
    L.orc_spectral_norm.argtypes = [ctypes.c_int, dp]
    L.orc_spectral_norm.restype = ctypes.c_double
    L.orc_carreau.argtypes = [pp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
    L.orc_carreau_lagged.argtypes = [pp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, dp, dp]
    L.orc_sc_force.argtypes = [pp, u8p, dp, dp]
    L.orc_charge_field.argtypes = [pp, u8p, dp, dp, dp, dp]
    L.orc_poisson_solve.argtypes = [pp, u8p, dp, dp, ctypes.c_double, dp,
                                    ctypes.POINTER(ctypes.c_int), dp]
    L.orc_poisson_system.argtypes = [pp, u8p, dp, dp, dp, dp,
                                     ctypes.POINTER(ctypes.c_long),
                                     ctypes.POINTER(ctypes.c_int)]
    L.orc_efield.argtypes = [pp, u8p, dp, dp]
    L.orc_stream.argtypes = [pp, u8p, dp, dp, dp, dp, dp, dp]
    L.orc_init.argtypes = [pp, u8p, dp, dp, dp, dp, dp, dp, dp]
    L.orc_apply_io.argtypes = [pp, u8p, dp, dp]
    L.orc_step.argtypes = [pp, u8p, dp, u8p, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_set_threads.restype = ctypes.c_int
    return L


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))


def make_params(cfg: dict) -> Params:
    """Map a workload parameter dictionary to the oracle's parameter struct."""
    P = Params()
    P.dim = cfg["dim"]
    P.nx, P.ny, P.nz = cfg["shape"]
    for i, v in enumerate(cfg["face_bc"]):
        P.face_bc[i] = _FACE[v]
    for i, v in enumerate(cfg["phi_bc"]):
        P.phi_bc[i] = _PHI[v]
    P.phi_axis = cfg["phi_axis"]
    P.charge_model = _CHARGE[cfg["charge_model"]]
    P.force_el = _FEL[cfg["force_el"]]
    P.neutralize = int(cfg["neutralize"])
    P.poisson_maxit = cfg["poisson_maxit"]
    P.poisson_fixed_sweeps = cfg["poisson_fixed_sweeps"]
    P.alpha_mode = _ALPHA[cfg["alpha_mode"]]
    P.eps_face = _EPS_FACE[cfg.get("eps_face", "arithmetic")]
    P.carreau_lagged = int(cfg.get("carreau_lagged", 0))
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
    return P


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's site-parallel loops (n <= 0 keeps the
    current setting); returns the number in use. Results do not depend on
    it: every global sum is taken serially in site order."""
    return int(lib().orc_set_threads(int(n)))


def Q_of(dim: int) -> int:
    return 9 if dim == 2 else 19


def lattice(dim: int):
    Q = Q_of(dim)
    c = (ctypes.c_int * (3 * Q))()
    w = np.zeros(Q)
    cs2 = ctypes.c_double()
    lib().orc_lattice(dim, c, _dp(w), ctypes.byref(cs2))
    return np.array(list(c), dtype=np.int64).reshape(Q, 3), w, cs2.value


def feq(dim, rho, u):
    out = np.zeros(Q_of(dim))
    u3 = np.zeros(3)
    u3[: len(u)] = u
    lib().orc_feq(dim, float(rho), _dp(u3), _dp(out))
    return out


def H(dim, f):
    return lib().orc_H(dim, _dp(np.ascontiguousarray(f, dtype=np.float64)))


def h(dim, f, d, a):
    return lib().orc_h(dim, _dp(np.ascontiguousarray(f, np.float64)),
                       _dp(np.ascontiguousarray(d, np.float64)), float(a))


def h_prime0(dim, f, d):
    return lib().orc_h_prime0(dim, _dp(np.ascontiguousarray(f, np.float64)),
                              _dp(np.ascontiguousarray(d, np.float64)))


def alpha(dim, f, d, eq_tol=1e-8):
    a = ctypes.c_double()
    st = lib().orc_alpha(dim, _dp(np.ascontiguousarray(f, np.float64)),
                         _dp(np.ascontiguousarray(d, np.float64)), float(eq_tol),
                         ctypes.cast(ctypes.pointer(a), ctypes.POINTER(ctypes.c_double)))
    return a.value, st


def alpha_bisect(dim, f, d):
    return lib().orc_alpha_bisect(dim, _dp(np.ascontiguousarray(f, np.float64)),
                                  _dp(np.ascontiguousarray(d, np.float64)))


def spectral_norm(dim, Pi):
    P = np.zeros((3, 3))
    P[:dim, :dim] = np.asarray(Pi)[:dim, :dim]
    return lib().orc_spectral_norm(dim, _dp(np.ascontiguousarray(P).reshape(-1)))


def carreau(cfg, Pn, a, rho):
    P = make_params(cfg)
    g = ctypes.c_double()
    nu = ctypes.c_double()
    dpt = ctypes.POINTER(ctypes.c_double)
    lib().orc_carreau(ctypes.byref(P), float(Pn), float(a), float(rho),
                      ctypes.cast(ctypes.pointer(g), dpt), ctypes.cast(ctypes.pointer(nu), dpt))
    return g.value, nu.value


def carreau_lagged(cfg, Pn, a, rho, nu_prev):
    """gdot and nu of the lagged Carreau reading (tau from nu_prev)."""
    P = make_params(cfg)
    g = ctypes.c_double()
    nu = ctypes.c_double()
    dpt = ctypes.POINTER(ctypes.c_double)
    lib().orc_carreau_lagged(ctypes.byref(P), float(Pn), float(a), float(rho), float(nu_prev),
                             ctypes.cast(ctypes.pointer(g), dpt), ctypes.cast(ctypes.pointer(nu), dpt))
    return g.value, nu.value


def _n(cfg):
    nx, ny, nz = cfg["shape"]
    return nx * ny * nz


def sc_force(cfg, mask, rho):
    P = make_params(cfg)
    F = np.zeros(3 * _n(cfg))
    lib().orc_sc_force(ctypes.byref(P), _u8(mask), _dp(rho), _dp(F))
    return F.reshape(-1, 3)


def charge_field(cfg, mask, rho):
    P = make_params(cfg)
    q = np.zeros(_n(cfg))
    K = np.zeros(_n(cfg))
    sums = np.zeros(2)
    lib().orc_charge_field(ctypes.byref(P), _u8(mask), _dp(rho), _dp(q), _dp(K), _dp(sums))
    return q, K, sums


def poisson_solve(cfg, mask, rho, qn, phi0=None, qmean=0.0):
    P = make_params(cfg)
    phi = np.zeros(_n(cfg)) if phi0 is None else np.array(phi0, dtype=np.float64)
    it = ctypes.c_int()
    res = ctypes.c_double()
    lib().orc_poisson_solve(ctypes.byref(P), _u8(mask), _dp(rho), _dp(qn), float(qmean), _dp(phi),
                            ctypes.byref(it),
                            ctypes.cast(ctypes.pointer(res), ctypes.POINTER(ctypes.c_double)))
    return phi, it.value, res.value


def poisson_system(cfg, mask, rho, qn):
    P = make_params(cfg)
    N = _n(cfg)
    n_unk = int(np.sum(mask != SOLID))
    A = np.zeros(n_unk * n_unk)
    b = np.zeros(n_unk)
    index = (ctypes.c_long * N)()
    nu = ctypes.c_int()
    lib().orc_poisson_system(ctypes.byref(P), _u8(mask), _dp(rho), _dp(qn), _dp(A), _dp(b),
                             index, ctypes.byref(nu))
    return A.reshape(n_unk, n_unk), b, np.array(list(index), dtype=np.int64)


def efield(cfg, mask, phi):
    P = make_params(cfg)
    E = np.zeros(3 * _n(cfg))
    lib().orc_efield(ctypes.byref(P), _u8(mask), _dp(phi), _dp(E))
    return E.reshape(-1, 3)


def stream(cfg, mask, fs, gs=None, u_in=None, rho=None):
    """Streaming alone: returns the populations after one streaming step."""
    P = make_params(cfg)
    N = _n(cfg)
    fs = np.ascontiguousarray(fs, dtype=np.float64).reshape(-1)
    out = np.zeros_like(fs)
    gout = None
    if gs is not None:
        gs = np.ascontiguousarray(gs, dtype=np.float64).reshape(-1)
        gout = np.zeros_like(gs)
    u_in = np.zeros(3 * N) if u_in is None else np.ascontiguousarray(u_in, np.float64).reshape(-1)
    rho = np.zeros(N) if rho is None else np.ascontiguousarray(rho, np.float64)
    lib().orc_stream(ctypes.byref(P), _u8(mask), _dp(u_in), _dp(rho), _dp(fs), _dp(gs),
                     _dp(out), _dp(gout))
    return out, gout


class Sim:
    """Stateful wrapper: populations f (post-streaming), g, phi."""

    def __init__(self, cfg: dict, fields: dict):
        self.cfg = cfg
        self.P = make_params(cfg)
        self.N = _n(cfg)
        self.Q = Q_of(cfg["dim"])
        mask = fields.get("mask")
        if mask is None:
            mask = np.zeros(self.N, np.uint8)
        self.mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        self.u_in = np.array(fields.get("u_in", np.zeros((self.N, 3))), dtype=np.float64).reshape(-1)
        # the adaptive inlet: the nozzle sites whose mean velocity rescales
        # the initial inlet profile each step
        reg = fields.get("inlet_region")
        self.region = None if reg is None else np.ascontiguousarray(reg, dtype=np.uint8).reshape(-1)
        self.u_in0 = self.u_in.copy() if self.region is not None else None
        rho0 = np.ascontiguousarray(fields["rho"], dtype=np.float64).reshape(-1)
        u0 = fields.get("u")
        u0 = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64).reshape(-1)
        q0 = fields.get("q")
        q0 = None if q0 is None else np.ascontiguousarray(q0, dtype=np.float64).reshape(-1)
        self.f = np.zeros(self.Q * self.N)
        self.transport = cfg["charge_model"] == "transport"
        self.g = np.zeros(7 * self.N) if self.transport else None
        self.phi = np.zeros(self.N)
        rc = lib().orc_init(ctypes.byref(self.P), _u8(self.mask), _dp(rho0), _dp(u0),
                            _dp(q0), _dp(self.u_in), _dp(self.f), _dp(self.g), _dp(self.phi))
        if rc != 0:
            raise ValueError(f"oracle rejected the parameters (code {rc})")
        if fields.get("f") is not None:
            self.f[:] = np.asarray(fields["f"], dtype=np.float64).reshape(-1)
            lib().orc_apply_io(ctypes.byref(self.P), _u8(self.mask), _dp(self.u_in), _dp(self.f))
        self.rho = np.zeros(self.N)
        self.u = np.zeros(3 * self.N)
        self.q = np.zeros(self.N)
        self.alpha = np.zeros(self.N)
        self.nu = np.zeros(self.N)
        self.diag = np.zeros(NDIAG)
        self.t = 0

    def step(self, n: int = 1):
        for _ in range(n):
            rc = lib().orc_step(ctypes.byref(self.P), _u8(self.mask), _dp(self.u_in),
                                None if self.region is None else _u8(self.region), _dp(self.u_in0),
                                _dp(self.f), _dp(self.g), _dp(self.phi), _dp(self.rho),
                                _dp(self.u), _dp(self.q), _dp(self.alpha), _dp(self.nu),
                                _dp(self.diag))
            if rc != 0:
                raise ValueError(f"oracle step failed (code {rc})")
            self.t += 1
        return dict(zip(DIAG_NAMES, self.diag.tolist()))

    def moments(self):
        """rho and rho*u of the current (post-streaming) populations."""
        c, _, _ = lattice(self.cfg["dim"])
        f = self.f.reshape(self.Q, self.N)
        return f.sum(0), f.T @ c.astype(np.float64)
