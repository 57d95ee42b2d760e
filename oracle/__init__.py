"""FP64 CPU oracle for the chemical-potential multiphase LBM step.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package's smoke check and
by the benchmark's CPU-baseline and reference legs, never by the product path.
It is a ctypes view of oracle/liboracle.so (plain C, FP64, no FMA contraction),
which shares no code with the CUDA library.

Functions that have no independent pin in the CPU tests are marked
"parity unpinned" in their docstring; every function here is currently
pinned (see tests/test_oracle_*.py).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

D2Q9, D3Q19 = 0, 1
SCHEMES = {"EFDS2": 0, "EFDS4": 1, "EFDS6": 2, "CFDS4": 3, "CFDS6": 4, "CFDS8": 5,
           "OCFDS4": 6, "E4": 7, "E8": 8}
COMPACT = ("CFDS4", "CFDS6", "CFDS8", "OCFDS4")
EXPLICIT_LINE = ("EFDS2", "EFDS4", "EFDS6")
OK, EINVAL, ENOMEM, EUNSTABLE = 0, -1, -2, -4

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class Params(C.Structure):
    _fields_ = [("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("Tr", C.c_double),
                ("k", C.c_double), ("kappa", C.c_double), ("tau", C.c_double), ("scheme", C.c_int),
                ("collision", C.c_int), ("mrt_s", C.c_double * 9), ("eos", C.c_int), ("acentric", C.c_double)]


class Obs(C.Structure):
    _fields_ = [("max_v", C.c_double), ("max_u", C.c_double), ("rho_center", C.c_double),
                ("rho_corner", C.c_double), ("mass", C.c_double), ("max_drho", C.c_double),
                ("step", C.c_longlong), ("status", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_cs_pressure.restype = C.c_double
        L.or_cs_pressure.argtypes = [C.c_double] * 5
        L.or_cs_mu.restype = C.c_double
        L.or_cs_mu.argtypes = [C.c_double] * 5
        L.or_cs_critical.argtypes = [C.c_double] * 3 + [_dp, _dp]
        L.or_maxwell.argtypes = [C.c_double] * 4 + [_dp, _dp]
        L.or_scheme_coeffs.argtypes = [C.c_int, _dp, _dp, _dp, _dp]
        L.or_deriv_line.argtypes = [C.c_int, _dp, C.c_int, _dp]
        L.or_deriv2_line.argtypes = [C.c_int, _dp, C.c_int, _dp]
        L.or_gradient.argtypes = [C.c_int] * 5 + [_dp, _dp]
        L.or_laplacian.argtypes = [C.c_int] * 5 + [_dp, _dp]
        L.or_lattice_q.argtypes = [C.c_int]
        L.or_lattice_e.argtypes = [C.c_int, _ip, _dp]
        L.or_feq.argtypes = [C.c_int, C.c_double, _dp, _dp]
        L.or_set_solid.argtypes = [C.c_void_p, C.c_void_p, C.c_double]
        L.or_solid_layers.argtypes = [C.c_void_p, C.c_void_p]
        L.or_eos_make.argtypes = [C.c_int] + [C.c_double] * 5 + [C.c_void_p]
        L.or_eos_pressure.argtypes = [C.c_void_p, C.c_double]
        L.or_eos_pressure.restype = C.c_double
        L.or_eos_mu.argtypes = [C.c_void_p, C.c_double]
        L.or_eos_mu.restype = C.c_double
        L.or_eos_maxwell.argtypes = [C.c_void_p, _dp, _dp]
        L.or_pr_alpha.argtypes = [C.c_double] * 3
        L.or_pr_alpha.restype = C.c_double
        L.or_pr_critical.argtypes = [C.c_double] * 3 + [_dp, _dp]
        L.or_cubic_critical.argtypes = [C.c_int] + [C.c_double] * 3 + [_dp, _dp]
        L.or_flat_profile.argtypes = [C.c_void_p, C.c_int, C.c_double, _dp, _dp]
        L.or_mrt_matrix.argtypes = [_dp]
        L.or_mrt_matrix.restype = None
        L.or_mrt_inverse.argtypes = [_dp]
        L.or_mrt_collide.argtypes = [_dp, _dp, _dp, _dp, _dp]
        L.or_mrt_collide.restype = None
        L.or_edm.argtypes = [C.c_int, C.c_double, _dp, _dp, _dp]
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.POINTER(Params)]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_init_droplet.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_init_slab.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_init_profile.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_int]
        L.or_set_f.argtypes = [C.c_void_p, _dp]
        L.or_get_f.argtypes = [C.c_void_p, _dp]
        L.or_get_density.argtypes = [C.c_void_p, _dp]
        L.or_get_fields.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.or_step.argtypes = [C.c_void_p, C.c_longlong]
        L.or_observables.argtypes = [C.c_void_p, C.POINTER(Obs)]
        L.or_temperature.restype = C.c_double
        L.or_temperature.argtypes = [C.c_void_p]
        L.or_mlp_forward.argtypes = [_ip, C.c_int, _dp, _dp, C.c_int, _dp, _dp]
        L.or_mlp_loss_grad.argtypes = [_ip, C.c_int, _dp, _dp, _dp, C.c_int, _dp, _dp]
        L.or_adam_step.argtypes = [C.c_int, _dp, _dp, _dp, _dp, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_int]
        _LIB = L
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _scheme(s):
    return SCHEMES[s] if isinstance(s, str) else int(s)


# ---------------------------------------------------------------- EOS
def cs_pressure(rho, a=1.0, b=4.0, R=1.0, T=0.07):
    return lib().or_cs_pressure(rho, a, b, R, T)


def cs_mu(rho, a=1.0, b=4.0, R=1.0, T=0.07):
    return lib().or_cs_mu(rho, a, b, R, T)


def cs_critical(a=1.0, b=4.0, R=1.0):
    rc, Tc = C.c_double(), C.c_double()
    if lib().or_cs_critical(a, b, R, C.byref(rc), C.byref(Tc)) != OK:
        raise ValueError("invalid CS constants")
    return rc.value, Tc.value


def maxwell(T, a=1.0, b=4.0, R=1.0):
    g, l = C.c_double(), C.c_double()
    rc = lib().or_maxwell(a, b, R, T, C.byref(g), C.byref(l))
    if rc != OK:
        raise ValueError("Maxwell construction failed (T >= Tc?)")
    return g.value, l.value


def maxwell_tr(Tr, a=1.0, b=4.0, R=1.0):
    return maxwell(Tr * cs_critical(a, b, R)[1], a, b, R)


# ---------------------------------------------------------------- differences
def scheme_coeffs(scheme):
    v = [C.c_double() for _ in range(4)]
    lib().or_scheme_coeffs(_scheme(scheme), *[C.byref(x) for x in v])
    return tuple(x.value for x in v)  # alpha, a, b, c


def deriv_line(scheme, f):
    f = _f64(f)
    d = np.empty_like(f)
    if lib().or_deriv_line(_scheme(scheme), _ptr(f), f.size, _ptr(d)) != OK:
        raise ValueError("bad scheme/size")
    return d


def deriv2_line(scheme, f):
    f = _f64(f)
    d = np.empty_like(f)
    if lib().or_deriv2_line(_scheme(scheme), _ptr(f), f.size, _ptr(d)) != OK:
        raise ValueError("bad scheme/size")
    return d


def gradient(scheme, phi):
    """phi: array shaped (ny, nx) or (nz, ny, nx); returns (dim, *phi.shape)."""
    phi = _f64(phi)
    dim = phi.ndim
    nz, ny, nx = (1,) + phi.shape if dim == 2 else phi.shape
    g = np.empty((dim,) + phi.shape)
    if lib().or_gradient(_scheme(scheme), dim, nx, ny, nz, _ptr(phi), _ptr(g)) != OK:
        raise ValueError("bad scheme/size")
    return g


def laplacian(scheme, phi):
    phi = _f64(phi)
    dim = phi.ndim
    nz, ny, nx = (1,) + phi.shape if dim == 2 else phi.shape
    out = np.empty_like(phi)
    if lib().or_laplacian(_scheme(scheme), dim, nx, ny, nz, _ptr(phi), _ptr(out)) != OK:
        raise ValueError("bad scheme/size")
    return out


# ---------------------------------------------------------------- lattice
def lattice(lat):
    q = lib().or_lattice_q(lat)
    e = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    lib().or_lattice_e(lat, e.ctypes.data_as(_ip), _ptr(w))
    return e, w


BGK, MRT = 0, 1
EOS_CS, EOS_PR, EOS_VDW, EOS_RKS = 0, 1, 2, 3


class Eos(C.Structure):
    _fields_ = [("kind", C.c_int), ("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("T", C.c_double),
                ("Tc", C.c_double), ("rho_c", C.c_double), ("alpha", C.c_double), ("rho_max", C.c_double)]


def eos_make(kind, a, b, R, Tr, acentric=0.344):
    """An equation of state (EOS_CS, or EOS_PR of Eq. 14-15) at T = Tr T_c."""
    e = Eos()
    if lib().or_eos_make(kind, a, b, R, Tr, acentric, C.byref(e)) != OK:
        raise ValueError("invalid EOS parameters")
    return e


def eos_pressure(e, rho):
    return lib().or_eos_pressure(C.byref(e), rho)


def eos_mu(e, rho):
    return lib().or_eos_mu(C.byref(e), rho)


def eos_maxwell(e):
    g, l = C.c_double(), C.c_double()
    if lib().or_eos_maxwell(C.byref(e), C.byref(g), C.byref(l)) != OK:
        raise ValueError("Maxwell construction failed")
    return g.value, l.value


def pr_alpha(T, Tc, acentric):
    return lib().or_pr_alpha(T, Tc, acentric)


def cubic_critical(kind, a, b, R):
    rc, Tc = C.c_double(), C.c_double()
    if lib().or_cubic_critical(kind, a, b, R, C.byref(rc), C.byref(Tc)) != OK:
        raise ValueError
    return rc.value, Tc.value


def flat_profile(n, y0, Tr, k, kappa, eos="CS", a=1.0, b=4.0, R=1.0, acentric=0.344):
    """Equilibrium flat interface (Eq. 29): (rho, drho/dy) at nodes 0..n-1."""
    p = Params(0, 8, 8, 1, a, b, R, Tr, k, kappa, 1.0, 0, 0, (C.c_double * 9)(),
               {"CS": EOS_CS, "PR": EOS_PR, "VDW": EOS_VDW, "RKS": EOS_RKS}[eos], acentric)
    rho, d = np.empty(n), np.empty(n)
    if lib().or_flat_profile(C.byref(p), n, y0, _ptr(rho), _ptr(d)) != OK:
        raise ValueError("invalid parameters")
    return rho, d


def pr_critical(a, b, R):
    rc, Tc = C.c_double(), C.c_double()
    if lib().or_pr_critical(a, b, R, C.byref(rc), C.byref(Tc)) != OK:
        raise ValueError
    return rc.value, Tc.value


def mrt_rates(tau):
    """The relaxation rates the paper chooses (Eq. 5 and the text after it)."""
    return [1.0, 1.64, 1.54, 1.0, 1.7, 1.0, 1.7, 1.0 / tau, 1.0 / tau]


def mrt_matrix():
    M = np.empty(81)
    lib().or_mrt_matrix(_ptr(M))
    return M.reshape(9, 9)


def mrt_inverse():
    M = np.empty(81)
    if lib().or_mrt_inverse(_ptr(M)) != OK:
        raise RuntimeError("singular")
    return M.reshape(9, 9)


def mrt_collide(f, feq_, Fi, s):
    out = np.empty(9)
    lib().or_mrt_collide(_ptr(_f64(f)), _ptr(_f64(feq_)), _ptr(_f64(Fi)), _ptr(_f64(s)), _ptr(out))
    return out


def feq(lat, rho, u):
    u = _f64(list(u) + [0.0] * (3 - len(u)))
    q = lib().or_lattice_q(lat)
    out = np.zeros(q)
    lib().or_feq(lat, rho, _ptr(u), _ptr(out))
    return out


def edm(lat, rho, u, F):
    u = _f64(list(u) + [0.0] * (3 - len(u)))
    F = _f64(list(F) + [0.0] * (3 - len(F)))
    q = lib().or_lattice_q(lat)
    out = np.zeros(q)
    lib().or_edm(lat, rho, _ptr(u), _ptr(F), _ptr(out))
    return out


# ---------------------------------------------------------------- simulation
class Sim:
    """One periodic droplet/slab simulation, plain FP64 (the paper's step)."""

    def __init__(self, lattice=D2Q9, nx=64, ny=64, nz=1, a=1.0, b=4.0, R=1.0, Tr=0.7, k=0.4,
                 kappa=1.0, tau=1.0, scheme="EFDS2", collision="BGK", mrt_s=None, eos="CS", acentric=0.344):
        """collision "MRT" (D2Q9): rates s_1..s_9 of Eq. 5, by default the
        paper's (1, 1.64, 1.54, 1, 1.7, 1, 1.7, 1/tau, 1/tau)."""
        if mrt_s is None:
            mrt_s = mrt_rates(tau)
        self.p = Params(lattice, nx, ny, nz, a, b, R, Tr, k, kappa, tau, _scheme(scheme),
                        {"BGK": BGK, "MRT": MRT}[collision], (C.c_double * 9)(*mrt_s),
                        {"CS": EOS_CS, "PR": EOS_PR, "VDW": EOS_VDW, "RKS": EOS_RKS}[eos], acentric)
        self.h = lib().or_create(C.byref(self.p))
        if not self.h:
            raise ValueError("invalid oracle parameters")
        self.q = lib().or_lattice_q(lattice)
        self.dim = 2 if lattice == D2Q9 else 3
        self.shape = (ny, nx) if self.dim == 2 else (nz, ny, nx)
        self.n = nx * ny * nz

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().or_destroy(h)
            self.h = None

    @property
    def T(self):
        return lib().or_temperature(self.h)

    def _check(self, rc):
        if rc not in (OK,):
            raise RuntimeError("oracle call failed: %d" % rc)

    def set_solid(self, mask, mu_w):
        """Wall nodes (Appendix A): mask of the lattice shape, wall chemical potential."""
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(-1))
        assert m.size == self.n
        if lib().or_set_solid(self.h, m.ctypes.data_as(C.c_void_p), mu_w) != OK:
            raise ValueError("walls need an explicit scheme (EFDS2/4/6) and a fluid node")

    def solid_layers(self):
        out = np.zeros(self.n, dtype=np.int32)
        lib().or_solid_layers(self.h, out.ctypes.data_as(C.c_void_p))
        return out.reshape(self.shape)

    def init_droplet(self, radius, width=10.0, center=None, rho_l=0.0, rho_g=0.0):
        c = _f64(center) if center is not None else None
        self._check(lib().or_init_droplet(self.h, _ptr(c) if c is not None else None, radius, width,
                                          rho_l, rho_g))

    def init_slab(self, axis, thickness, width=10.0, rho_l=0.0, rho_g=0.0):
        self._check(lib().or_init_slab(self.h, axis, thickness, width, rho_l, rho_g))

    def init_profile(self, r, rho, center=None):
        r, rho = _f64(r), _f64(rho)
        c = _f64(center) if center is not None else None
        self._check(lib().or_init_profile(self.h, _ptr(c) if c is not None else None, _ptr(r), _ptr(rho),
                                          r.size))

    def set_f(self, f):
        f = _f64(f).reshape(self.q, self.n)
        self._check(lib().or_set_f(self.h, _ptr(f)))

    def get_f(self):
        f = np.empty((self.q,) + self.shape)
        lib().or_get_f(self.h, _ptr(f))
        return f

    def density(self):
        r = np.empty(self.shape)
        lib().or_get_density(self.h, _ptr(r))
        return r

    def fields(self):
        rho = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        F = np.empty((3,) + self.shape)
        mu = np.empty(self.shape)
        rc = lib().or_get_fields(self.h, _ptr(rho), _ptr(u), _ptr(F), _ptr(mu))
        if rc != OK:
            raise RuntimeError("oracle fields failed: %d" % rc)
        return {"rho": rho, "u": u[: self.dim], "F": F[: self.dim], "mu": mu}

    def step(self, n=1):
        return lib().or_step(self.h, n)

    def observables(self):
        o = Obs()
        lib().or_observables(self.h, C.byref(o))
        return o.as_dict()


# ---------------------------------------------------------------- MLP
def _sizes(sizes):
    return np.ascontiguousarray(sizes, dtype=np.int32)


def mlp_param_count(sizes):
    return sum(sizes[l + 1] * sizes[l] + sizes[l + 1] for l in range(len(sizes) - 1))


def mlp_forward(sizes, params, x):
    s = _sizes(sizes)
    params, x = _f64(params), _f64(x)
    batch = x.shape[0]
    y = np.empty((batch, sizes[-1]))
    lib().or_mlp_forward(s.ctypes.data_as(_ip), len(sizes) - 1, _ptr(params), _ptr(x), batch, _ptr(y), None)
    return y


def mlp_loss_grad(sizes, params, x, target):
    s = _sizes(sizes)
    params, x, target = _f64(params), _f64(x), _f64(target)
    grad = np.empty_like(params)
    loss = C.c_double()
    rc = lib().or_mlp_loss_grad(s.ctypes.data_as(_ip), len(sizes) - 1, _ptr(params), _ptr(x), _ptr(target),
                                x.shape[0], C.byref(loss), _ptr(grad))
    if rc != OK:
        raise ValueError("bad MLP arguments")
    return loss.value, grad


def adam_step(params, m, v, grad, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on float64 arrays params, m, v."""
    for a in (params, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(grad)
    lib().or_adam_step(params.size, _ptr(params), _ptr(m), _ptr(v), _ptr(g), lr, beta1, beta2, eps, t)
