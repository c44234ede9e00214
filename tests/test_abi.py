"""CPU tests of the C ABI: the library loads and exports every entry point include/lbm.h
declares; host-side argument validation and the Section 4.2 unit scaling (no GPU needed)."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle import thermo as th
from paper_1909_12390_gb300 import build as lbm_build
from paper_1909_12390_gb300 import lbm


@pytest.fixture(scope="module")
def lib():
    lbm_build.build()
    return lbm.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_entry_point(lib):
    declared = _declared()
    assert "lbm_create" in declared and "lbm_step" in declared and "lbm_fields" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(lbm.EXPORTS) <= set(declared)


@pytest.mark.parametrize("bad", [
    dict(shape=(8, 8), tau=0.5), dict(shape=(8, 8), tau=0.4), dict(shape=(0, 8)),
    dict(shape=(8, 8), gamma=[0.0, 1.0]), dict(shape=(8, 8), G=0.0),
    dict(shape=(8, 8), collision=lbm.MRT), dict(shape=(8, 8), kij=[[0, 0.1], [0.2, 0]]),
    dict(shape=(8, 8), precision=7), dict(shape=(8, 8), T=-1.0),
    dict(shape=(8, 8), collision=lbm.MRT, mrt_rates=[1.0] * 8 + [2.5]),
    dict(comps=[(0.07, -0.06, 0.3, 1.0), (0.09, 0.05, 0.2, 2.0)]),
])
def test_invalid_arguments_rejected_before_any_device_work(lib, bad):
    kw = dict(shape=(8, 8), comps=[(0.07, 0.06, 0.3, 1.0), (0.09, 0.05, 0.2, 2.0)], T=0.06, tau=1.0,
              gamma=[0.5, 1.0])
    kw.update(bad)
    comps = kw.pop("comps")
    shape = kw.pop("shape")
    with pytest.raises(lbm.LBMError) as ei:
        lbm.Lattice(shape, comps, **kw)
    assert ei.value.status == lbm.ERR_ARG


def test_nc_limit_and_d2q9_nz(lib):
    comps = [(0.07, 0.06, 0.3, 1.0)] * 5
    with pytest.raises(lbm.LBMError) as ei:
        lbm.Lattice((8, 8), comps, T=0.06, tau=1.0)
    assert ei.value.status == lbm.ERR_ARG
    g = lbm.Grid(8, 8, 2, 9)
    import ctypes
    h = ctypes.c_void_p()
    c = (lbm.Component * 1)(lbm.Component(0.07, 0.06, 0.3, 1.0))
    e = lbm.Eos(T=0.06, beta=1.0, G=-1.0)
    assert lib.lbm_create(ctypes.byref(g), 1, c, ctypes.byref(e), 1.0, ctypes.byref(h)) == lbm.ERR_ARG
    assert b"nz" in lib.lbm_last_error(None)


def test_scale_to_lattice_matches_section_4_2(lib):
    phys = [(666.06, 616.0, 0.1522, 44.097), (845.8, 488.6, 0.2514, 72.15)]
    got, T, p = lbm.scale_to_lattice(phys, 666.06, 200.0)
    want, ts, ps = th.lattice_components([th.Component("a", *phys[0]), th.Component("b", *phys[1])])
    for g, w in zip(got, want):
        assert g[0] == pytest.approx(w.Tc, rel=1e-14)
        assert g[1] == pytest.approx(w.pc, rel=1e-14)
        assert g[3] == pytest.approx(w.M, rel=1e-14)
    assert T == pytest.approx(666.06 * ts, rel=1e-14)
    assert p == pytest.approx(200.0 * ps, rel=1e-14)


def test_flash_rejects_bad_arguments_before_any_device_work():
    """lbm_flash validates on the host and returns LBM_ERR_ARG without touching the GPU."""
    from paper_1909_12390_gb300 import lbm
    comps = [(0.0729, 0.0596, 0.011, 1.0), (0.163, 0.049, 0.2, 3.62)]
    bad = [
        dict(T=[0.1], p=[0.05], z=[[0.5, 0.6]]),                      # z does not sum to 1
        dict(T=[-0.1], p=[0.05], z=[[0.5, 0.5]]),                     # T <= 0
        dict(T=[0.1], p=[0.05], z=[[0.5, 0.5]], kij=[[[0, 0.1], [0.2, 0]]]),  # asymmetric
    ]
    for kw in bad:
        with pytest.raises(lbm.LBMError) as ei:
            lbm.flash(comps, **kw)
        assert ei.value.status == lbm.ERR_ARG
    with pytest.raises(lbm.LBMError) as ei:
        lbm.flash(comps * 3, [0.1], [0.05], [[1.0 / 6] * 6])          # nc > 4
    assert ei.value.status == lbm.ERR_ARG
    r = lbm.flash(comps, [], [], np.zeros((0, 2)))                     # no cases: nothing to do
    assert r["V"].shape == (0,)


def test_binding_constants_equal_the_header():
    """Every enumerator and numeric #define of include/lbm.h that the Python binding repeats
    (LBM_X -> lbm.X) has the header's value, and the status codes and step paths are all
    repeated."""
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"\bLBM_([A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    consts.update({m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+LBM_([A-Z0-9_]+)\s+(-?\d+)", src)})
    for name in ("OK", "ERR_ARG", "ERR_CUDA", "ERR_OOM", "ERR_PSI_DOMAIN", "ERR_NONFINITE", "ERR_TIMEOUT",
                 "PATH_AUTO", "PATH_TWO_KERNEL", "PATH_FUSED", "PATH_TRAILING", "PATH_QUEUE"):
        assert name in consts and hasattr(lbm, name), name
    checked = [n for n in consts if hasattr(lbm, n)]
    assert len(checked) >= 20
    for name in checked:
        assert getattr(lbm, name) == consts[name], name
