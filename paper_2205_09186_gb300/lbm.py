"""ctypes binding of include/lbm.h (argument marshalling only).

Every function of the C ABI is exposed under the same name.  PyTorch provides
device memory (through an lbm_allocator backed by its caching allocator) and
the CUDA stream; all arithmetic runs in liblbm.so.  Importing this module on
a machine without the built library raises ImportError: there is no CPU path.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ENOTSUP, LBM_ESCRATCH = (
    0, -1, -2, -3, -4, -5, -6, -7)
LBM_D2Q9, LBM_D3Q19 = 0, 1
LBM_EOS_CS, LBM_EOS_PR, LBM_EOS_VDW, LBM_EOS_RKS = 0, 1, 2, 3
EOS = {"CS": LBM_EOS_CS, "PR": LBM_EOS_PR, "VDW": LBM_EOS_VDW, "RKS": LBM_EOS_RKS}
SCHEMES = {"EFDS2": 0, "EFDS4": 1, "EFDS6": 2, "CFDS4": 3, "CFDS6": 4, "CFDS8": 5, "OCFDS4": 6, "E4": 7, "E8": 8}
LBM_FP64, LBM_FP32DEV = 0, 1
LBM_BGK, LBM_MRT = 0, 1


class lbm_params(C.Structure):
    _fields_ = [("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("eos", C.c_int),
                ("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("Tr", C.c_double),
                ("k", C.c_double), ("kappa", C.c_double), ("tau", C.c_double),
                ("scheme", C.c_int), ("precision", C.c_int), ("mu_fp64", C.c_int), ("rho_ref", C.c_double),
                ("collision", C.c_int), ("mrt_s", C.c_double * 9), ("acentric", C.c_double)]


class lbm_obs(C.Structure):
    _fields_ = [("max_v", C.c_double), ("max_u", C.c_double), ("rho_center", C.c_double),
                ("rho_corner", C.c_double), ("mass", C.c_double), ("max_drho", C.c_double),
                ("step", C.c_longlong), ("status", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class lbm_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_h = C.c_void_p

# name -> (restype, argtypes); every entry point declared in include/lbm.h
SIGNATURES = {
    "lbm_create": (C.c_int, [C.POINTER(lbm_params), C.c_void_p, C.POINTER(lbm_allocator), C.POINTER(C.c_void_p)]),
    "lbm_destroy": (None, [_h]),
    "lbm_init_droplet": (C.c_int, [_h, _dp, C.c_double, C.c_double, C.c_double, C.c_double]),
    "lbm_init_slab": (C.c_int, [_h, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]),
    "lbm_init_profile": (C.c_int, [_h, _dp, _dp, _dp, C.c_int]),
    "lbm_init_density": (C.c_int, [_h, _dp]),
    "lbm_set_f": (C.c_int, [_h, _dp]),
    "lbm_step": (C.c_int, [_h, C.c_longlong]),
    "lbm_step_timed": (C.c_int, [_h, C.c_longlong, _dp]),
    "lbm_observables": (C.c_int, [_h, C.POINTER(lbm_obs)]),
    "lbm_step_observe": (C.c_int, [_h, C.c_longlong, C.POINTER(lbm_obs)]),
    "lbm_step_observe_async": (C.c_int, [_h, C.c_longlong, C.c_void_p]),
    "lbm_get_density": (C.c_int, [_h, _dp]),
    "lbm_get_f": (C.c_int, [_h, _dp]),
    "lbm_get_force": (C.c_int, [_h, _dp, _dp]),
    "lbm_get_step": (C.c_longlong, [_h]),
    "lbm_device_state": (C.c_int, [_h, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "lbm_critical": (C.c_int, [C.c_double, C.c_double, C.c_double, _dp, _dp]),
    "lbm_maxwell": (C.c_int, [C.POINTER(lbm_params), _dp, _dp]),
    "lbm_eos_critical": (C.c_int, [C.POINTER(lbm_params), _dp, _dp]),
    "lbm_flat_profile": (C.c_int, [C.POINTER(lbm_params), C.c_int, C.c_double, _dp, _dp]),
    "lbm_force_angle": (C.c_int, [_h, _dp, C.c_double, _dp]),
    "lbm_set_solid": (C.c_int, [_h, C.POINTER(C.c_ubyte), C.c_double]),
    "lbm_bulk_mu": (C.c_int, [C.POINTER(lbm_params), C.c_double, _dp]),
    "lbm_lattice_q": (C.c_int, [C.c_int]),
    "lbm_set_zchunk": (C.c_int, [_h, C.c_int]),
    "lbm_set_tile_rows": (C.c_int, [_h, C.c_int]),
    "lbm_autotune": (C.c_int, [_h, C.POINTER(C.c_int)]),
    "lbm_strerror": (C.c_char_p, [C.c_int]),
    "lbm_observables_noalloc": (C.c_int, [C.POINTER(lbm_params), C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong,
                                          C.c_longlong, C.c_void_p, C.POINTER(lbm_obs)]),
    "lbm_batch_create": (C.c_int, [C.POINTER(lbm_params), C.c_int, C.c_void_p, C.POINTER(lbm_allocator),
                                   C.POINTER(C.c_void_p)]),
    "lbm_batch_destroy": (None, [_h]),
    "lbm_batch_init_droplets": (C.c_int, [_h, _dp, C.c_double]),
    "lbm_batch_step": (C.c_int, [_h, C.c_longlong]),
    "lbm_batch_observables": (C.c_int, [_h, C.POINTER(lbm_obs)]),
    "lbm_batch_get_density": (C.c_int, [_h, C.c_int, _dp]),
    "lbm_batch_get_step": (C.c_longlong, [_h]),
    "lbm_batch_size": (C.c_int, [_h, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lbm_batch_inject_stall": (C.c_int, [_h, C.c_int]),
    "lbm_batch_set_tiles": (C.c_int, [_h, C.c_int]),
    "lbm_batch_autotune": (C.c_int, [_h, C.c_int, C.POINTER(C.c_int)]),
    "lbm_mlp_create": (C.c_int, [C.POINTER(C.c_int), C.c_int, C.c_int, C.c_void_p, C.POINTER(lbm_allocator),
                                 C.POINTER(C.c_void_p)]),
    "lbm_mlp_destroy": (None, [_h]),
    "lbm_mlp_param_count": (C.c_longlong, [_h]),
    "lbm_mlp_set_params": (C.c_int, [_h, _fp]),
    "lbm_mlp_get_params": (C.c_int, [_h, _fp]),
    "lbm_mlp_forward": (C.c_int, [_h, _fp, C.c_int, _fp]),
    "lbm_mlp_loss_grad": (C.c_int, [_h, _fp, _fp, C.c_int, _fp, _fp]),
    "lbm_mlp_set_data": (C.c_int, [_h, _fp, _fp, C.c_int]),
    "lbm_mlp_train": (C.c_int, [_h, C.c_int, C.c_float, _fp]),
}

_LIB = None


def lib():
    """Load liblbm.so (built by paper_2205_09186_gb300.build); no fallback."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("liblbm.so is not built (run __graft_entry__.build()); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


class LBMError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (%d)" % (what, lib().lbm_strerror(code).decode(), code))
        self.code = code


def check(rc, what):
    if rc != LBM_OK:
        raise LBMError(rc, what)
    return rc


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_params(lattice=LBM_D2Q9, nx=64, ny=64, nz=1, a=1.0, b=4.0, R=1.0, Tr=0.7, k=0.25, kappa=0.1, tau=1.0,
                scheme="EFDS2", precision=LBM_FP64, mu_fp64=0, rho_ref=0.0, collision=LBM_BGK, mrt_s=None,
                eos=LBM_EOS_CS, acentric=0.344):
    """collision: LBM_BGK / LBM_MRT or "BGK" / "MRT"; mrt_s None = the paper's rates;
    eos: LBM_EOS_* or "CS" / "PR" / "VDW" / "RKS" (a, b, R are that EOS's constants)."""
    e = EOS[eos] if isinstance(eos, str) else int(eos)
    s = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    col = {"BGK": LBM_BGK, "MRT": LBM_MRT}[collision] if isinstance(collision, str) else int(collision)
    rates = (C.c_double * 9)(*(mrt_s if mrt_s is not None else [0.0] * 9))
    return lbm_params(lattice, nx, ny, nz, e, a, b, R, Tr, k, kappa, tau, s, precision, int(mu_fp64), rho_ref,
                      col, rates, acentric)


def lbm_bulk_mu(params, rho):
    """k^2 psi'(rho): the chemical potential of a uniform fluid of density rho."""
    out = C.c_double()
    check(lib().lbm_bulk_mu(C.byref(params), float(rho), C.byref(out)), "lbm_bulk_mu")
    return out.value


def lbm_observables_noalloc(params, d_f, d_rho, d_rho_prev=None, steps_since_prev=0, step=0, stream=None):
    """Observables of a caller-held device state; the library allocates nothing.
    Returns (status code, observables dict)."""
    o = lbm_obs()
    st = C.c_void_p(int(stream)) if stream is not None else None
    rc = lib().lbm_observables_noalloc(C.byref(params), C.c_void_p(d_f), C.c_void_p(d_rho),
                                       C.c_void_p(d_rho_prev) if d_rho_prev else None, steps_since_prev, step, st,
                                       C.byref(o))
    return rc, o.as_dict()


def lbm_critical(a=1.0, b=4.0, R=1.0):
    rc, Tc = C.c_double(), C.c_double()
    check(lib().lbm_critical(a, b, R, C.byref(rc), C.byref(Tc)), "lbm_critical")
    return rc.value, Tc.value


def lbm_eos_critical(params):
    rc, Tc = C.c_double(), C.c_double()
    check(lib().lbm_eos_critical(C.byref(params), C.byref(rc), C.byref(Tc)), "lbm_eos_critical")
    return rc.value, Tc.value


def lbm_flat_profile(params, n, y0):
    """(rho, drho/dy) of the equilibrium flat interface at nodes 0..n-1."""
    rho, d = np.empty(n), np.empty(n)
    check(lib().lbm_flat_profile(C.byref(params), n, y0, _ptr(rho), _ptr(d)), "lbm_flat_profile")
    return rho, d


def lbm_maxwell(params):
    g, l = C.c_double(), C.c_double()
    check(lib().lbm_maxwell(C.byref(params), C.byref(g), C.byref(l)), "lbm_maxwell")
    return g.value, l.value


class TorchAllocator:
    """lbm_allocator backed by PyTorch's CUDA caching allocator."""

    def __init__(self, device=None, stream=None):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = stream

        def _alloc(nbytes, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
            except Exception:  # out of memory -> NULL -> LBM_ENOMEM
                return None

        def _free(ptr, nbytes, ctx):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.struct = lbm_allocator(self._a, self._f, None)


class Sim:
    """One periodic simulation handle (C ABI: lbm_create ... lbm_destroy)."""

    def __init__(self, params=None, stream=None, allocator="torch", **kw):
        self.params = params if params is not None else make_params(**kw)
        self.Q = lib().lbm_lattice_q(self.params.lattice)
        self.D = 2 if self.params.lattice == LBM_D2Q9 else 3
        p = self.params
        self.shape = (p.ny, p.nx) if self.D == 2 else (p.nz, p.ny, p.nx)
        self.N = p.nx * p.ny * p.nz
        st = None
        self._alloc = None
        if stream is not None:
            st = C.c_void_p(int(stream))
        if allocator == "torch":
            import torch
            if stream is None:
                st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
            self._alloc = TorchAllocator(stream=torch.cuda.current_stream() if stream is None else None)
        h = C.c_void_p()
        check(lib().lbm_create(C.byref(p), st, C.byref(self._alloc.struct) if self._alloc else None, C.byref(h)),
              "lbm_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def lbm_init_droplet(self, radius, width=10.0, center=None, rho_l=0.0, rho_g=0.0):
        c = _f64(center) if center is not None else None
        return check(lib().lbm_init_droplet(self.h, _ptr(c) if c is not None else None, radius, width, rho_l, rho_g),
                     "lbm_init_droplet")

    def lbm_init_slab(self, axis, thickness, width=10.0, rho_l=0.0, rho_g=0.0):
        return check(lib().lbm_init_slab(self.h, axis, thickness, width, rho_l, rho_g), "lbm_init_slab")

    def lbm_init_profile(self, r, rho, center=None):
        r, rho = _f64(r), _f64(rho)
        c = _f64(center) if center is not None else None
        return check(lib().lbm_init_profile(self.h, _ptr(c) if c is not None else None, _ptr(r), _ptr(rho), r.size),
                     "lbm_init_profile")

    def lbm_init_density(self, rho):
        rho = _f64(rho).reshape(-1)
        assert rho.size == self.N
        return check(lib().lbm_init_density(self.h, _ptr(rho)), "lbm_init_density")

    def lbm_set_f(self, f):
        f = _f64(f).reshape(-1)
        assert f.size == self.Q * self.N
        return check(lib().lbm_set_f(self.h, _ptr(f)), "lbm_set_f")

    def lbm_step(self, n=1):
        return check(lib().lbm_step(self.h, n), "lbm_step")

    def lbm_step_timed(self, n=1):
        ms = np.zeros(3)
        check(lib().lbm_step_timed(self.h, n, _ptr(ms)), "lbm_step_timed")
        return ms

    def lbm_observables(self, raise_unstable=False):
        o = lbm_obs()
        rc = lib().lbm_observables(self.h, C.byref(o))
        if rc not in (LBM_OK, LBM_EUNSTABLE) or (raise_unstable and rc == LBM_EUNSTABLE):
            check(rc, "lbm_observables")
        return o.as_dict()

    def lbm_step_observe(self, n=1, raise_unstable=False):
        o = lbm_obs()
        rc = lib().lbm_step_observe(self.h, n, C.byref(o))
        if rc not in (LBM_OK, LBM_EUNSTABLE) or (raise_unstable and rc == LBM_EUNSTABLE):
            check(rc, "lbm_step_observe")
        return o.as_dict()

    def lbm_step_observe_async(self, n, out_addr):
        """n steps; the observables of the state the last one started from are
        written, by the stream, to the lbm_obs at address out_addr (page-locked
        host or device memory), valid after the next synchronisation; read
        them with lbm_obs.from_address(out_addr)."""
        check(lib().lbm_step_observe_async(self.h, n, C.c_void_p(out_addr)), "lbm_step_observe_async")

    def lbm_force_angle(self, frac=0.1, center=None):
        """(max angle, |F|-weighted mean angle, nodes) of Eq. 30 on the current state."""
        out = np.zeros(3)
        c = _f64(center) if center is not None else None
        check(lib().lbm_force_angle(self.h, _ptr(c) if c is not None else None, frac, _ptr(out)), "lbm_force_angle")
        return out[0], out[1], int(out[2])

    def lbm_set_solid(self, mask, mu_w=0.0):
        """Wall nodes (Appendix A) where `mask` (lattice shape) is nonzero,
        with wall chemical potential mu_w; mask None removes the walls."""
        if mask is None:
            check(lib().lbm_set_solid(self.h, None, 0.0), "lbm_set_solid")
            return
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        if m.size != int(np.prod(self.shape)):
            raise ValueError("mask must have the lattice's size")
        check(lib().lbm_set_solid(self.h, m.ctypes.data_as(C.POINTER(C.c_ubyte)), float(mu_w)), "lbm_set_solid")

    def lbm_get_density(self, out=None):
        """Density field as FP64 host array; `out` (e.g. a pinned buffer of
        self.shape or its size, C-contiguous float64) receives it in place."""
        if out is None:
            out = np.empty(self.shape)
        elif out.dtype != np.float64 or out.size != int(np.prod(self.shape)) or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float64 array of the lattice size")
        check(lib().lbm_get_density(self.h, _ptr(out)), "lbm_get_density")
        return out

    def lbm_get_f(self):
        out = np.empty((self.Q,) + self.shape)
        check(lib().lbm_get_f(self.h, _ptr(out)), "lbm_get_f")
        return out

    def lbm_get_force(self):
        F = np.empty((self.D,) + self.shape)
        mu = np.empty(self.shape)
        check(lib().lbm_get_force(self.h, _ptr(F), _ptr(mu)), "lbm_get_force")
        return F, mu

    def lbm_get_step(self):
        return lib().lbm_get_step(self.h)

    def lbm_set_zchunk(self, zc):
        return check(lib().lbm_set_zchunk(self.h, zc), "lbm_set_zchunk")

    def lbm_set_tile_rows(self, rows_per_thread):
        return check(lib().lbm_set_tile_rows(self.h, int(rows_per_thread)), "lbm_set_tile_rows")

    def lbm_autotune(self):
        """z chunk (D3Q19) or tile rows per thread (D2Q9 split step) chosen by
        timing; 0 if nothing to tune.  The state is left undefined."""
        zc = C.c_int()
        check(lib().lbm_autotune(self.h, C.byref(zc)), "lbm_autotune")
        return zc.value

    def lbm_device_state(self):
        f, r = C.c_void_p(), C.c_void_p()
        check(lib().lbm_device_state(self.h, C.byref(f), C.byref(r)), "lbm_device_state")
        return f.value, r.value


class Batch:
    """Many D2Q9 droplets advanced together (C ABI: lbm_batch_*)."""

    def __init__(self, params_list, stream=None, allocator="torch"):
        import torch
        n = len(params_list)
        arr = (lbm_params * n)(*params_list)
        self.params = list(params_list)
        st = C.c_void_p(int(stream)) if stream is not None else C.c_void_p(torch.cuda.current_stream().cuda_stream)
        self._alloc = TorchAllocator(stream=torch.cuda.current_stream()) if allocator == "torch" else None
        h = C.c_void_p()
        check(lib().lbm_batch_create(arr, n, st, C.byref(self._alloc.struct) if self._alloc else None, C.byref(h)),
              "lbm_batch_create")
        self.h = h
        self.n = n

    def close(self):
        if getattr(self, "h", None):
            lib().lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def lbm_batch_init_droplets(self, radius, width=10.0):
        r = _f64(radius)
        assert r.size == self.n
        return check(lib().lbm_batch_init_droplets(self.h, _ptr(r), width), "lbm_batch_init_droplets")

    def lbm_batch_step(self, n=1):
        return check(lib().lbm_batch_step(self.h, n), "lbm_batch_step")

    def lbm_batch_observables(self, raise_errors=True):
        out = (lbm_obs * self.n)()
        rc = lib().lbm_batch_observables(self.h, out)
        if raise_errors and rc != LBM_OK:
            check(rc, "lbm_batch_observables")
        return rc, [o.as_dict() for o in out]

    def lbm_batch_get_density(self, c):
        p = self.params[c]
        out = np.empty((p.ny, p.nx))
        check(lib().lbm_batch_get_density(self.h, c, _ptr(out)), "lbm_batch_get_density")
        return out

    def lbm_batch_get_step(self):
        return lib().lbm_batch_get_step(self.h)

    def lbm_batch_size(self):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        check(lib().lbm_batch_size(self.h, C.byref(a), C.byref(b), C.byref(c)), "lbm_batch_size")
        return a.value, b.value, c.value

    def lbm_batch_inject_stall(self, cta):
        return check(lib().lbm_batch_inject_stall(self.h, cta), "lbm_batch_inject_stall")

    def lbm_batch_set_tiles(self, rows_per_thread):
        return check(lib().lbm_batch_set_tiles(self.h, int(rows_per_thread)), "lbm_batch_set_tiles")

    def lbm_batch_autotune(self, steps=5, cache=None):
        """Tile rows per thread (1, 2, 4) chosen by timing; the tuning steps
        advance the state (initialise before tuning, and again afterwards).  cache: path of a JSON file
        of earlier choices keyed by the device and the cases' shapes; a hit
        sets that choice without timing, a miss records the new one."""
        key = None
        if cache is not None:
            import hashlib
            import json
            import os
            import torch
            shapes = [(p.nx, p.ny, p.scheme, p.precision, p.mu_fp64, p.collision) for p in self.params]
            key = hashlib.sha1(json.dumps([torch.cuda.get_device_name(), shapes]).encode()).hexdigest()
            table = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    table = json.load(f)
            if key in table:
                self.lbm_batch_set_tiles(table[key])
                return table[key]
        r = C.c_int()
        check(lib().lbm_batch_autotune(self.h, int(steps), C.byref(r)), "lbm_batch_autotune")
        if key is not None:
            table[key] = r.value
            with open(cache, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
        return r.value


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _fptr(a):
    return a.ctypes.data_as(_fp)


class MLP:
    """Warm-start network (C ABI: lbm_mlp_*)."""

    def __init__(self, sizes, max_batch, stream=None, allocator="torch"):
        import torch
        sz = (C.c_int * len(sizes))(*sizes)
        self.sizes = list(sizes)
        st = C.c_void_p(int(stream)) if stream is not None else C.c_void_p(torch.cuda.current_stream().cuda_stream)
        self._alloc = TorchAllocator(stream=torch.cuda.current_stream()) if allocator == "torch" else None
        h = C.c_void_p()
        check(lib().lbm_mlp_create(sz, len(sizes) - 1, max_batch, st,
                                   C.byref(self._alloc.struct) if self._alloc else None, C.byref(h)), "lbm_mlp_create")
        self.h = h
        self.nparam = lib().lbm_mlp_param_count(h)

    def close(self):
        if getattr(self, "h", None):
            lib().lbm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def lbm_mlp_set_params(self, p):
        p = _f32(p)
        assert p.size == self.nparam
        return check(lib().lbm_mlp_set_params(self.h, _fptr(p)), "lbm_mlp_set_params")

    def lbm_mlp_get_params(self):
        out = np.empty(self.nparam, dtype=np.float32)
        check(lib().lbm_mlp_get_params(self.h, _fptr(out)), "lbm_mlp_get_params")
        return out

    def lbm_mlp_forward(self, x):
        x = _f32(x)
        y = np.empty((x.shape[0], self.sizes[-1]), dtype=np.float32)
        check(lib().lbm_mlp_forward(self.h, _fptr(x), x.shape[0], _fptr(y)), "lbm_mlp_forward")
        return y

    def lbm_mlp_loss_grad(self, x, t):
        x, t = _f32(x), _f32(t)
        g = np.empty(self.nparam, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        check(lib().lbm_mlp_loss_grad(self.h, _fptr(x), _fptr(t), x.shape[0], _fptr(loss), _fptr(g)),
              "lbm_mlp_loss_grad")
        return float(loss[0]), g

    def lbm_mlp_set_data(self, x, t):
        x, t = _f32(x), _f32(t)
        return check(lib().lbm_mlp_set_data(self.h, _fptr(x), _fptr(t), x.shape[0]), "lbm_mlp_set_data")

    def lbm_mlp_train(self, iters, lr=1e-3):
        loss = np.zeros(1, dtype=np.float32)
        check(lib().lbm_mlp_train(self.h, iters, lr, _fptr(loss)), "lbm_mlp_train")
        return float(loss[0])
