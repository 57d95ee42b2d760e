"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, and
exports every entry point declared in include/lbm.h (no GPU calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(lbm_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    import paper_2205_09186_gb300 as pkg
    return pkg.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2205_09186_gb300 import lbm
    assert set(declared_functions()) <= set(lbm.SIGNATURES)


def test_host_only_entry_points(libpath):
    # the EOS helpers of the C ABI run on the host and need no GPU
    from paper_2205_09186_gb300 import lbm
    import oracle as O
    rc, Tc = lbm.lbm_critical()
    orc, oTc = O.cs_critical()
    assert abs(rc - orc) < 1e-12 and abs(Tc - oTc) < 1e-14
    for tr in (0.9, 0.7, 0.5, 0.3, 0.2):
        g, l = lbm.lbm_maxwell(lbm.make_params(Tr=tr))
        og, ol = O.maxwell_tr(tr)
        assert abs(g / og - 1) < 1e-9 and abs(l / ol - 1) < 1e-12
    # Peng-Robinson (Eq. 14-15, the paper's a = 2/49, b = 2/21, acentric 0.344)
    A, B = 2.0 / 49.0, 2.0 / 21.0
    rc, Tc = lbm.lbm_eos_critical(lbm.make_params(eos="PR", a=A, b=B, Tr=0.7))
    orc, oTc = O.pr_critical(A, B, 1.0)
    assert abs(rc / orc - 1) < 1e-12 and abs(Tc / oTc - 1) < 1e-12
    for tr in (0.9, 0.7, 0.5):
        g, l = lbm.lbm_maxwell(lbm.make_params(eos="PR", a=A, b=B, Tr=tr))
        og, ol = O.eos_maxwell(O.eos_make(O.EOS_PR, A, B, 1.0, tr, 0.344))
        assert abs(g / og - 1) < 1e-9 and abs(l / ol - 1) < 1e-12
    for name, kind, a in (("VDW", O.EOS_VDW, 9.0 / 49.0), ("RKS", O.EOS_RKS, 2.0 / 49.0)):
        q = lbm.make_params(eos=name, a=a, b=B, Tr=0.7)
        assert np.allclose(lbm.lbm_eos_critical(q), O.cubic_critical(kind, a, B, 1.0), rtol=1e-12, atol=0)
        assert np.allclose(lbm.lbm_maxwell(q), O.eos_maxwell(O.eos_make(kind, a, B, 1.0, 0.7, 0.344)),
                           rtol=1e-9, atol=0)
    assert lbm.lib().lbm_lattice_q(0) == 9 and lbm.lib().lbm_lattice_q(1) == 19
    assert lbm.lib().lbm_strerror(-4).decode().startswith("simulation unstable")


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2205_09186_gb300 import lbm
    monkeypatch.setattr(lbm, "_LIB", None)
    monkeypatch.setattr(lbm, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        lbm.lib()


def test_flat_profile_matches_oracle(libpath):
    # the library's analytic flat interface (Eq. 29) against the oracle's, two
    # independent quadratures of the same first integral; CS and PR
    import numpy as np
    from paper_2205_09186_gb300 import lbm
    import oracle as O
    for kw, okw in ((dict(Tr=0.6, k=0.4, kappa=0.1), dict()),
                    (dict(eos="PR", a=2.0 / 49.0, b=2.0 / 21.0, Tr=0.7, k=0.2, kappa=0.01),
                     dict(eos="PR", a=2.0 / 49.0, b=2.0 / 21.0))):
        r, d = lbm.lbm_flat_profile(lbm.make_params(**kw), 96, 47.5)
        ro, do = O.flat_profile(96, 47.5, kw["Tr"], kw["k"], kw["kappa"], **okw)
        assert np.max(np.abs(r - ro)) < 1e-8 * np.max(ro)
        assert np.max(np.abs(d - do)) < 5e-8 * np.max(do)


def test_bulk_mu_matches_oracle(libpath):
    # k^2 psi'(rho) of the library's host EOS against the oracle's, for each EOS
    from paper_2205_09186_gb300 import lbm
    import oracle as O
    k = 0.3
    cases = [("CS", O.EOS_CS, 1.0, 4.0, (0.01, 0.1, 0.5)),
             ("PR", O.EOS_PR, 2.0 / 49.0, 2.0 / 21.0, (0.05, 1.0, 6.0)),
             ("VDW", O.EOS_VDW, 9.0 / 49.0, 2.0 / 21.0, (0.05, 1.0, 6.0)),
             ("RKS", O.EOS_RKS, 2.0 / 49.0, 2.0 / 21.0, (0.05, 1.0, 6.0))]
    for name, kind, a, b, rhos in cases:
        p = lbm.make_params(eos=name, a=a, b=b, Tr=0.8, k=k)
        e = O.eos_make(kind, a, b, 1.0, 0.8, 0.344)
        for rho in rhos:
            assert lbm.lbm_bulk_mu(p, rho) == pytest.approx(k * k * O.eos_mu(e, rho), rel=1e-12, abs=1e-14)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_bulk_mu(lbm.make_params(), -1.0)
