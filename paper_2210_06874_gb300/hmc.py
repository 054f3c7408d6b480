"""ctypes binding of the C ABI in include/hmc.h (argument marshalling only).

Every function here checks tensor shapes, dtypes and devices, passes raw
device pointers and the current CUDA stream to libhmc_gb300.so and turns a
non-zero hmc_status into HmcError.  No step of the method runs in Python:
there is no CPU fallback, and importing this module on a machine without the
built library raises.

Field layouts (torch tensors on the context's CUDA device, contiguous):
    phi, F, pi      float64  [Nt, V]
    psi (FP64)      complex128 [Nt, V]
    psi (MIXED)     complex64  [Nt, V]
"""
import ctypes
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhmc_gb300.so")

HMC_OK = 0
HMC_ERR_BAD_ARG = -1
HMC_ERR_CUDA = -2
HMC_ERR_CG_NOT_CONVERGED = -3
HMC_ERR_NONFINITE = -4
HMC_ERR_TIMEOUT = -5
HMC_ERR_UNSUPPORTED = -6
STATUS_NAMES = {
    0: "HMC_OK", -1: "HMC_ERR_BAD_ARG", -2: "HMC_ERR_CUDA", -3: "HMC_ERR_CG_NOT_CONVERGED",
    -4: "HMC_ERR_NONFINITE", -5: "HMC_ERR_TIMEOUT", -6: "HMC_ERR_UNSUPPORTED",
}
PREC_FP64 = 0
PREC_MIXED = 1


class HmcError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__("%s failed: %s (%d)" % (fn, STATUS_NAMES.get(code, "?"), code))
        self.code = code


class hmc_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("Nt", ctypes.c_int), ("kappa", ctypes.c_double),
                ("U", ctypes.c_double), ("beta", ctypes.c_double), ("n_md", ctypes.c_int),
                ("traj_length", ctypes.c_double), ("cg_tol", ctypes.c_double),
                ("cg_max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("ru_delta", ctypes.c_double), ("team_ctas", ctypes.c_int),
                ("tile_slices", ctypes.c_int), ("inner_ctas", ctypes.c_int),
                ("operand_mode", ctypes.c_int), ("cluster_mode", ctypes.c_int),
                ("integrator", ctypes.c_int), ("mu", ctypes.c_double),
                ("ru_every", ctypes.c_int), ("hb_gamma", ctypes.c_double),
                ("hb_inner", ctypes.c_int)]


class hmc_cg_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("status", ctypes.c_int),
                ("fp64_iterations", ctypes.c_int)]


class hmc_traj_out(ctypes.Structure):
    _fields_ = [("dH", ctypes.c_double), ("H0", ctypes.c_double), ("H1", ctypes.c_double),
                ("u", ctypes.c_double), ("accept", ctypes.c_int),
                ("cg_iterations", ctypes.c_int), ("cg_solves", ctypes.c_int),
                ("reliable_updates", ctypes.c_int), ("max_true_residual", ctypes.c_double),
                ("status", ctypes.c_int), ("fp64_iterations", ctypes.c_int),
                ("cg_iterations_outer", ctypes.c_int), ("cg_solves_outer", ctypes.c_int)]


_lib = None

# symbol -> (restype, argtypes); mirrors include/hmc.h
_P = ctypes.c_void_p
SIGNATURES = {
    "hmc_ctx_create": (ctypes.c_int, [ctypes.POINTER(hmc_params), ctypes.POINTER(_P)]),
    "hmc_ctx_destroy": (ctypes.c_int, [_P]),
    "hmc_get_transfer_matrix": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "hmc_apply_M": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, _P]),
    "hmc_apply_Mdag": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, _P]),
    "hmc_cg_solve": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, ctypes.POINTER(hmc_cg_stats), _P]),
    "hmc_force": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "hmc_action": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "hmc_trajectory": (ctypes.c_int, [_P, _P, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_uint32, ctypes.POINTER(hmc_traj_out), _P]),
    "hmc_rng_draw": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                    ctypes.c_uint32, ctypes.c_int64, _P, _P, _P, _P]),
    "hmc_version": (ctypes.c_char_p, []),
    "hmc_batch_create": (ctypes.c_int, [ctypes.POINTER(hmc_params), ctypes.c_int,
                                        ctypes.POINTER(_P)]),
    "hmc_batch_destroy": (ctypes.c_int, [_P]),
    "hmc_batch_layout": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int]),
    "hmc_batch_trajectory": (ctypes.c_int, [_P, _P, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.POINTER(hmc_traj_out), _P]),
    "hmc_brs_phases": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
    "hmc_apply_brs": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P, _P,
                                     ctypes.c_int, ctypes.c_int, _P]),
    "hmc_correlator_k0": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         _P, ctypes.POINTER(hmc_cg_stats), _P]),
    "hmc_spin_traces": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, _P,
                                       ctypes.POINTER(hmc_cg_stats), _P]),
    "hmc_cg_solve_noalloc": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                            ctypes.c_double, ctypes.c_int,
                                            ctypes.POINTER(hmc_cg_stats), _P]),
    "hmc_ctx_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_double]),
    "hmc_debug_team_padding": (ctypes.c_int, [_P, ctypes.c_int]),
}


def load_library(path=LIB_PATH):
    """Load libhmc_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libhmc_gb300.so is missing at %s: run "
                           "`python -m paper_2210_06874_gb300.build_lib` first" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(fn, code, allow=()):
    if code != HMC_OK and code not in allow:
        raise HmcError(fn, code)
    return code


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class Params:
    L: int
    Nt: int
    kappa: float = 1.0
    U: float = 2.0
    beta: float = 2.0
    n_md: int = 10
    traj_length: float = 1.0
    cg_tol: float = 1e-12
    cg_max_iter: int = 100000
    precision: int = PREC_FP64
    ru_delta: float = 0.0
    team_ctas: int = 0
    tile_slices: int = 0
    inner_ctas: int = 0
    operand_mode: int = 0
    cluster_mode: int = 0
    integrator: int = 0
    mu: float = 0.0
    ru_every: int = 0
    hb_gamma: float = 0.0
    hb_inner: int = 0

    @property
    def V(self):
        return 2 * self.L * self.L

    @property
    def delta(self):
        return self.beta / self.Nt

    def to_c(self):
        return hmc_params(self.L, self.Nt, self.kappa, self.U, self.beta, self.n_md,
                          self.traj_length, self.cg_tol, self.cg_max_iter, self.precision,
                          self.ru_delta, self.team_ctas, self.tile_slices,
                          self.inner_ctas, self.operand_mode, self.cluster_mode,
                          self.integrator, self.mu, self.ru_every, self.hb_gamma,
                          self.hb_inner)


class Context:
    """Owns an hmc_ctx (E, its FP16 split, workspaces) on the current device."""

    def __init__(self, params: Params):
        self.lib = load_library()
        self.params = params
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        cp = params.to_c()
        _check("hmc_ctx_create", self.lib.hmc_ctx_create(ctypes.byref(cp), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.hmc_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- checks ------------------------------------------------------------
    @property
    def shape(self):
        return (self.params.Nt, self.params.V)

    def _field(self, t, name, dtype):
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != dtype \
                or tuple(t.shape) != self.shape or not t.is_contiguous():
            raise ValueError("%s must be a contiguous %s tensor of shape %s on %s"
                             % (name, dtype, self.shape, self.device))
        return t

    # -- entry points --------------------------------------------------------
    def transfer_matrix(self):
        V = self.params.V
        out = torch.empty((V, V), dtype=torch.float64)
        _check("hmc_get_transfer_matrix",
               self.lib.hmc_get_transfer_matrix(self._h, _ptr(out), V * V))
        return out

    def _apply(self, fn, phi, psi, out, prec):
        dt = torch.complex128 if prec == PREC_FP64 else torch.complex64
        self._field(phi, "phi", torch.float64)
        self._field(psi, "psi", dt)
        if out is None:
            out = torch.empty_like(psi)
        self._field(out, "out", dt)
        _check(fn, getattr(self.lib, fn)(self._h, _ptr(phi), _ptr(psi), _ptr(out), prec,
                                         _stream()))
        return out

    def apply_M(self, phi, psi, out=None, prec=PREC_FP64):
        return self._apply("hmc_apply_M", phi, psi, out, prec)

    def apply_Mdag(self, phi, psi, out=None, prec=PREC_FP64):
        return self._apply("hmc_apply_Mdag", phi, psi, out, prec)

    def cg_solve(self, phi, chi, tol=None, max_iter=None, prec=PREC_FP64, x=None,
                 allow_not_converged=False):
        self._field(phi, "phi", torch.float64)
        self._field(chi, "chi", torch.complex128)
        if x is None:
            x = torch.empty_like(chi)
        self._field(x, "x", torch.complex128)
        st = hmc_cg_stats()
        tol = self.params.cg_tol if tol is None else tol
        max_iter = self.params.cg_max_iter if max_iter is None else max_iter
        allow = (HMC_ERR_CG_NOT_CONVERGED,) if allow_not_converged else ()
        _check("hmc_cg_solve", self.lib.hmc_cg_solve(self._h, _ptr(phi), _ptr(chi), _ptr(x),
                                                     tol, max_iter, prec, ctypes.byref(st),
                                                     _stream()), allow)
        return x, st

    def correlator_k0(self, phi, tol=None, max_iter=None, prec=PREC_FP64):
        """Zero-momentum single-particle correlator on sublattice A,
        C[t] (complex128 [Nt]) from one M^{-1} source (hmc_correlator_k0)."""
        self._field(phi, "phi", torch.float64)
        C = torch.empty(self.params.Nt, dtype=torch.complex128, device=phi.device)
        st = hmc_cg_stats()
        tol = self.params.cg_tol if tol is None else tol
        max_iter = self.params.cg_max_iter if max_iter is None else max_iter
        _check("hmc_correlator_k0",
               self.lib.hmc_correlator_k0(self._h, _ptr(phi), tol, max_iter, prec, _ptr(C),
                                          ctypes.byref(st), _stream()))
        return C, st

    def spin_traces(self, phi, n_noise, seed, chain=0, tol=None, max_iter=None,
                    prec=PREC_FP64):
        """Z2-noise estimates of the staggered spin traces (hmc_spin_traces):
        per-sample values complex128 [n_noise, 3] (T_s, T_u, T_ss), their
        means with chi_s appended (complex128 [4]) and the summed CG stats."""
        self._field(phi, "phi", torch.float64)
        samples = torch.empty(n_noise, 3, dtype=torch.complex128, device=phi.device)
        mean = torch.empty(4, dtype=torch.complex128, device=phi.device)
        st = hmc_cg_stats()
        tol = self.params.cg_tol if tol is None else tol
        max_iter = self.params.cg_max_iter if max_iter is None else max_iter
        _check("hmc_spin_traces",
               self.lib.hmc_spin_traces(self._h, _ptr(phi), int(n_noise), int(seed), int(chain),
                                        tol, max_iter, prec, _ptr(samples), _ptr(mean),
                                        ctypes.byref(st), _stream()))
        return samples, mean, st

    def force(self, phi, x, F=None):
        self._field(phi, "phi", torch.float64)
        self._field(x, "x", torch.complex128)
        if F is None:
            F = torch.empty_like(phi)
        self._field(F, "F", torch.float64)
        _check("hmc_force", self.lib.hmc_force(self._h, _ptr(phi), _ptr(x), _ptr(F), _stream()))
        return F

    def action(self, phi, chi, x):
        """S = sum(phi^2)/(2 delta U) + Re(chi^dag x) (FP64, host float)."""
        self._field(phi, "phi", torch.float64)
        self._field(chi, "chi", torch.complex128)
        self._field(x, "x", torch.complex128)
        out = ctypes.c_double()
        _check("hmc_action", self.lib.hmc_action(self._h, _ptr(phi), _ptr(chi), _ptr(x),
                                                 ctypes.byref(out), _stream()))
        return out.value

    def set_wait_limit(self, seconds):
        """Time limit of every bounded device wait of later launches (0: the
        default, 20 s)."""
        _check("hmc_ctx_set_wait_limit", self.lib.hmc_ctx_set_wait_limit(self._h, seconds))

    def debug_team_padding(self, extra_ctas):
        """Testing only: team barriers of later launches expect extra_ctas
        CTAs beyond those launched, so their bounded waits run out."""
        _check("hmc_debug_team_padding", self.lib.hmc_debug_team_padding(self._h, extra_ctas))

    def trajectory(self, phi, seed, traj_index, chain=0, allow_not_converged=False):
        self._field(phi, "phi", torch.float64)
        out = hmc_traj_out()
        allow = (HMC_ERR_CG_NOT_CONVERGED,) if allow_not_converged else ()
        _check("hmc_trajectory", self.lib.hmc_trajectory(self._h, _ptr(phi), seed, traj_index,
                                                         chain, ctypes.byref(out), _stream()),
               allow)
        return out


def brs_phases(L, Nt, phi):
    """exp(i phi) tables (complex128, complex64) for apply_brs (Eq. (2.2))."""
    lib = load_library()
    V = 2 * L * L
    if phi.dtype != torch.float64 or tuple(phi.shape) != (Nt, V) or not phi.is_contiguous():
        raise ValueError("phi must be contiguous float64 [Nt, V]")
    c64 = torch.empty((Nt, V), dtype=torch.complex128, device=phi.device)
    c32 = torch.empty((Nt, V), dtype=torch.complex64, device=phi.device)
    _check("hmc_brs_phases", lib.hmc_brs_phases(L, Nt, _ptr(phi), _ptr(c64), _ptr(c32),
                                                _stream()))
    return c64, c32


def apply_brs(L, Nt, delta_kappa, cis, psi, out=None, dagger=False):
    """M psi (or M^dag psi) of Eq. (2.2); complex128 -> FP64, complex64 -> FP32."""
    lib = load_library()
    V = 2 * L * L
    prec = PREC_FP64 if psi.dtype == torch.complex128 else PREC_MIXED
    for t in (cis, psi):
        if t.dtype != psi.dtype or tuple(t.shape) != (Nt, V) or not t.is_contiguous():
            raise ValueError("cis and psi must be contiguous [Nt, V] of the same complex dtype")
    if out is None:
        out = torch.empty_like(psi)
    elif out.dtype != psi.dtype or tuple(out.shape) != (Nt, V) or not out.is_contiguous():
        raise ValueError("out must be contiguous [Nt, V] of psi's dtype")
    _check("hmc_apply_brs", lib.hmc_apply_brs(L, Nt, delta_kappa, _ptr(cis), _ptr(psi),
                                              _ptr(out), prec, int(bool(dagger)), _stream()))
    return out


class Batch:
    """Many independent chains (one hmc_params each, MIXED precision) advanced
    by one persistent launch per trajectory (hmc_batch_*)."""

    def __init__(self, params_list):
        self.lib = load_library()
        self.params = list(params_list)
        self.n = len(self.params)
        arr = (hmc_params * self.n)(*[p.to_c() for p in self.params])
        h = ctypes.c_void_p()
        _check("hmc_batch_create", self.lib.hmc_batch_create(arr, self.n, ctypes.byref(h)))
        self._h = h
        off = (ctypes.c_int64 * (self.n + 1))()
        _check("hmc_batch_layout", self.lib.hmc_batch_layout(self._h, off, self.n + 1))
        self.offsets = [int(v) for v in off]
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.hmc_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def total(self):
        return self.offsets[-1]

    def view(self, phi, i):
        """Chain i's field [Nt, V] inside the packed tensor phi."""
        p = self.params[i]
        return phi[self.offsets[i]:self.offsets[i + 1]].view(p.Nt, p.V)

    def trajectory(self, phi, seed, traj_index, allow_failure=False):
        if not isinstance(phi, torch.Tensor) or phi.dtype != torch.float64 or \
                phi.device != self.device or phi.numel() != self.total or \
                not phi.is_contiguous():
            raise ValueError("phi must be a contiguous float64 tensor of %d elements on %s"
                             % (self.total, self.device))
        outs = (hmc_traj_out * self.n)()
        code = self.lib.hmc_batch_trajectory(self._h, _ptr(phi), seed, traj_index, outs,
                                             _stream())
        if not allow_failure:
            _check("hmc_batch_trajectory", code)
        return list(outs)


def rng_draw(seed, stream_id, traj, chain, n, device=None):
    """Philox draws of the library's generator: (raw uint32 [n,4], z0, z1)."""
    lib = load_library()
    device = device or torch.device("cuda", torch.cuda.current_device())
    raw = torch.empty((n, 4), dtype=torch.int32, device=device)
    z0 = torch.empty(n, dtype=torch.float64, device=device)
    z1 = torch.empty(n, dtype=torch.float64, device=device)
    _check("hmc_rng_draw", lib.hmc_rng_draw(seed, stream_id, traj, chain, n, _ptr(raw),
                                            _ptr(z0), _ptr(z1), _stream()))
    return raw, z0, z1


def check_noalloc_args(E, L, Nt, phi, chi, x, device):
    """Argument checks of cg_solve_noalloc, made before the library is called:
    E float64 [V, V], phi float64 [Nt, V], chi and x complex128 [Nt, V], all
    contiguous tensors on `device`, x not overlapping chi.  Raises ValueError."""
    if not (isinstance(L, int) and isinstance(Nt, int)) or L < 1 or Nt < 1:
        raise ValueError("L and Nt must be positive integers")
    V = 2 * L * L
    want = {"E": (E, torch.float64, (V, V)), "phi": (phi, torch.float64, (Nt, V)),
            "chi": (chi, torch.complex128, (Nt, V)), "x": (x, torch.complex128, (Nt, V))}
    for name, (t, dt, shape) in want.items():
        if not isinstance(t, torch.Tensor) or t.dtype != dt or tuple(t.shape) != shape \
                or not t.is_contiguous() or t.device != device:
            raise ValueError("%s must be a contiguous %s tensor of shape %s on %s"
                             % (name, dt, shape, device))
    if x.data_ptr() < chi.data_ptr() + chi.numel() * chi.element_size() and \
            chi.data_ptr() < x.data_ptr() + x.numel() * x.element_size():
        raise ValueError("x must not overlap chi")


def cg_solve_noalloc(E, L, Nt, phi, chi, x, tol, max_iter):
    """hmc_cg_solve_noalloc: FP64 CG with the library's static scratch (no
    device allocation inside the call).  E: float64 [V, V], phi: float64
    [Nt, V], chi and x: complex128 [Nt, V], all contiguous on the current
    CUDA device; x is written.  Returns (code, hmc_cg_stats)."""
    check_noalloc_args(E, L, Nt, phi, chi, x,
                       torch.device("cuda", torch.cuda.current_device()))
    lib = load_library()
    st = hmc_cg_stats()
    code = lib.hmc_cg_solve_noalloc(_ptr(E), L, Nt, _ptr(phi), _ptr(chi), _ptr(x), tol,
                                    max_iter, ctypes.byref(st), _stream())
    return code, st


def version():
    return load_library().hmc_version().decode()
