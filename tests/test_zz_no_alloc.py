"""The non-allocating observables entry point (lbm_observables_noalloc).

Callers that own every device buffer (an embedding application under a fixed
memory budget, or code where a new cudaMalloc would stall or fail) pass their
state as device pointers; the library keeps the reduction's partial results in
a fixed device array instead of allocating.  This test calls it through the C
ABI twice in a row on the state of a normal handle and checks it against the
allocating lbm_observables within the tolerance of the other parity tests.
It sits in its own file, collected last, and passes alone or after the rest."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09186_gb300 as pkg
    pkg.build()
    from paper_2205_09186_gb300 import lbm
    return lbm


KEYS = ("max_v", "max_u", "mass", "rho_center", "rho_corner")


class _DeviceArray:
    """A library-owned device buffer seen by torch (no copy)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2}


@pytest.mark.parametrize("lattice,shape,precision,scheme", [
    (0, (72, 40, 1), 0, "EFDS6"),
    (1, (40, 36, 44), 1, "EFDS6"),
    (1, (24, 24, 24), 0, "E4"),
])
def test_noalloc_matches_allocating_observables(L, lattice, shape, precision, scheme):
    import torch
    nx, ny, nz = shape
    p = L.make_params(lattice=lattice, nx=nx, ny=ny, nz=nz, Tr=0.8, k=0.25, kappa=0.1, scheme=scheme,
                      precision=precision)
    s = L.Sim(p)
    s.lbm_init_droplet(8.0)
    s.lbm_step(20)
    ref = s.lbm_observables()
    d_f, d_rho = s.lbm_device_state()
    stream = torch.cuda.current_stream().cuda_stream
    # FP64: the same kernels, so equal to rounding.  FP32 deviations: the handle
    # evaluates D3Q19 observables from its mu field (separate FP32 pass), this
    # entry point inside its tile kernel, so FP32 rounding differs.
    tol = 1e-12 if precision == 0 else 2e-6
    for _ in range(2):  # two calls in a row share the fixed array
        rc, o = L.lbm_observables_noalloc(s.params, d_f, d_rho, step=20, stream=stream)
        assert rc == L.LBM_OK and o["status"] == 0 and o["step"] == 20
        for k in KEYS:
            assert o[k] == pytest.approx(ref[k], rel=tol, abs=1e-300), k
    # max_drho against an earlier density held by the caller (here the same field)
    rc, o = L.lbm_observables_noalloc(s.params, d_f, d_rho, d_rho_prev=d_rho, steps_since_prev=5, step=20,
                                      stream=stream)
    assert rc == L.LBM_OK and o["max_drho"] == 0.0


@pytest.mark.parametrize("lattice,shape,precision", [
    (0, (72, 40, 1), 0), (0, (72, 40, 1), 1), (1, (40, 36, 44), 0), (1, (40, 36, 44), 1),
])
def test_noalloc_max_drho_against_earlier_density(L, lattice, shape, precision):
    # the caller keeps a copy of the density at step 20, runs 5 more steps and
    # asks for max |rho(25) - rho(20)| / 5; the handle's own lbm_observables,
    # whose previous observation was at step 20, reports the same quantity
    import torch
    nx, ny, nz = shape
    p = L.make_params(lattice=lattice, nx=nx, ny=ny, nz=nz, Tr=0.8, k=0.25, kappa=0.1, scheme="EFDS6",
                      precision=precision)
    s = L.Sim(p)
    s.lbm_init_droplet(8.0)
    s.lbm_step(20)
    s.lbm_observables()  # the handle's snapshot at step 20
    _, d_rho20 = s.lbm_device_state()
    n = nx * ny * nz
    # the caller's own copy of the stored density field (device to device)
    stored = torch.as_tensor(_DeviceArray(d_rho20, n, "<f8" if precision == 0 else "<f4"), device="cuda")
    prev = stored.clone()
    stream = torch.cuda.current_stream()
    s.lbm_step(5)
    ref = s.lbm_observables()
    assert ref["step"] == 25 and ref["max_drho"] > 0
    d_f, d_rho = s.lbm_device_state()
    for _ in range(2):
        rc, o = L.lbm_observables_noalloc(s.params, d_f, d_rho, d_rho_prev=prev.data_ptr(), steps_since_prev=5,
                                          step=25, stream=stream.cuda_stream)
        assert rc == L.LBM_OK and o["status"] == 0
        if precision == 0:
            assert o["max_drho"] == pytest.approx(ref["max_drho"], rel=1e-12)
        else:
            # the same float pairs differenced; the passes round the maxima
            # alike up to the FP32 rounding of one density value over dt
            assert abs(o["max_drho"] - ref["max_drho"]) <= 1e-6 * ref["rho_center"] / 5


def test_noalloc_rejects_oversized_and_compact(L):
    p = L.make_params(lattice=L.LBM_D2Q9, nx=8192, ny=8192, Tr=0.8, scheme="EFDS4")
    rc, _ = L.lbm_observables_noalloc(p, 1 << 20, 1 << 20)
    assert rc == L.LBM_ESCRATCH
    p = L.make_params(lattice=L.LBM_D2Q9, nx=64, ny=64, Tr=0.8, scheme="OCFDS4")
    rc, _ = L.lbm_observables_noalloc(p, 1 << 20, 1 << 20)
    assert rc == L.LBM_ENOTSUP
