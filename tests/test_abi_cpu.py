"""CPU checks of the C ABI: the library loads and exports every declared symbol; its host-only FP64
functions (correction coefficients, growth fit, argument validation) agree with the oracle."""
import math
import os
import re

import numpy as np
import pytest
from pathlib import Path

import oracle as O
from oracle.fit import growth_rate

P = pytest.importorskip("paper_1401_0838_gb300")
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def _declared():
    names = set()
    for fn in os.listdir(HEADER):
        if fn.endswith(".h"):
            txt = open(os.path.join(HEADER, fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(pic_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = P.lib()
    declared = _declared()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(P.EXPORTS) == declared


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("alpha", [0.1, 0.25, 0.3, 0.45, 0.55, 0.6, 0.7])
def test_coefficients_match_oracle(scheme, alpha):
    pe, pb = P.pic_compute_correction_coeffs(scheme, alpha)
    st, oe, ob = O.rational_coeffs(scheme, alpha)
    assert st == 0
    # two different solvers (QR here, Gaussian elimination in the oracle) of a system with
    # condition ~1e8: agreement to ~1e-16 * cond
    np.testing.assert_allclose(pe, oe, rtol=2e-7, atol=2e-8)
    np.testing.assert_allclose(pb, ob, rtol=2e-7, atol=2e-8)
    # the multiplier they interpolate agrees to 1e-10 everywhere on [0, 1]
    xi = np.linspace(0, 1, 101)
    r1 = np.polyval(pe[::-1], xi) / np.polyval(pb[::-1], xi)
    r2 = np.polyval(oe[::-1], xi) / np.polyval(ob[::-1], xi)
    assert np.abs(r1 - r2).max() < 1e-9


def test_coefficients_degenerate_and_errors():
    pe, pb = P.pic_compute_correction_coeffs(1, 0.5)
    assert list(pe) == [1, 0, 0, 0, 0] and list(pb) == [1, 0, 0, 0, 0]
    with pytest.raises(P.PicError) as e:
        P.pic_compute_correction_coeffs(0, -0.1)
    assert e.value.code == P.PIC_E_ARG
    with pytest.raises(P.PicError):
        P.pic_compute_correction_coeffs(7, 0.5)


def test_momentum_multiplier_coefficients():
    # Eq. 5 is also interpolated (host only); its ratio reproduces the nine nodes
    pe, pb = P.pic_compute_correction_coeffs(2, 0.5)
    for j in range(9):
        xi = j / 8
        m = O.multiplier(2, 0.5, math.asin(math.sqrt(xi)))
        assert abs(np.polyval(pe[::-1], xi) / np.polyval(pb[::-1], xi) - m) < 1e-10


@pytest.mark.parametrize("seed", range(4))
def test_growth_fit_matches_oracle(seed):
    rng = np.random.default_rng(seed)
    t = np.arange(150) * 0.7
    g = rng.uniform(0.01, 0.05)
    w = 1e-8 * (1 + 0.2 * rng.random(150)) + 1e-10 * np.exp(2 * g * t)
    w = np.minimum(w, 10 ** rng.uniform(-2, 3))
    a = P.pic_fit_growth_rate(t, w)
    b = growth_rate(t, w)
    assert a[1:] == b[1:]
    assert abs(a[0] - b[0]) < 1e-12 * abs(b[0])


def test_growth_fit_indices_refer_to_the_callers_arrays():
    # samples with w <= 0 or non-finite w are skipped by both fits; the window's indices still point
    # into the arrays passed in, so t[i0] and t[i1] are its first and last times
    t = np.arange(150) * 0.7
    w = 1e-8 * (1 + 0.2 * np.random.default_rng(3).random(150)) + 1e-10 * np.exp(0.06 * t)
    w = np.minimum(w, 1.0)
    ref = growth_rate(t, w)
    holes = w.copy()
    holes[[0, 7, 40, 41]] = (0.0, -1.0, np.nan, np.inf)
    a, b = P.pic_fit_growth_rate(t, holes), growth_rate(t, holes)
    assert a[1:] == b[1:]
    assert abs(a[0] - b[0]) < 1e-12 * abs(b[0])
    assert 41 < b[1] and b[2] == ref[2]  # same window end; no skipped sample inside the window
    assert holes[b[1]] > 0 and holes[b[2]] > 0


@pytest.mark.parametrize("bad", ["repeat", "decrease", "nan"])
def test_growth_fit_rejects_a_bad_time_axis(bad):
    t = np.arange(50) * 0.5
    w = np.exp(0.1 * t)
    if bad == "repeat":
        t[10] = t[9]
    elif bad == "decrease":
        t = t[::-1].copy()
    else:
        t[3] = np.nan
    with pytest.raises(P.PicError) as e:
        P.pic_fit_growth_rate(t, w)
    assert e.value.code == P.PIC_E_ARG
    with pytest.raises(ValueError):
        growth_rate(t, w)


def test_create_validates_before_touching_the_gpu():
    cfg = P.pic_config_default(dt=0.71)  # 2D Courant limit 1/sqrt(2)
    with pytest.raises(P.PicError) as e:
        P.pic_create(cfg)
    assert e.value.code == P.PIC_E_CFL
    cfg = P.pic_config_default(ndim=4)
    with pytest.raises(P.PicError) as e:
        P.pic_create(cfg)
    assert e.value.code == P.PIC_E_ARG
    cfg = P.pic_config_default(ndim=3, nx=8, ny=8, nz=8, dt=0.58)  # 3D limit 1/sqrt(3)
    with pytest.raises(P.PicError) as e:
        P.pic_create(cfg)
    assert e.value.code == P.PIC_E_CFL
    # sizes whose slot count would overflow the library's int arithmetic are refused up front
    for kw in (dict(ppc_per_species=(1 << 20) + 1), dict(bin_capacity=(1 << 24) + 1), dict(ppc_per_species=-1)):
        with pytest.raises(P.PicError) as e:
            P.pic_create(P.pic_config_default(**kw))
        assert e.value.code == P.PIC_E_ARG, kw


def test_create_validates_the_ck_solver():
    # CK (2D): stable while dt^2 max(1/dx^2, 1/dz^2, (1-4bx)/dx^2 + (1-4bz)/dz^2) < 1, i.e. dt < 1 at
    # beta = 1/8, dx = dz = 1; 3D and weights outside [0, 1/4] are rejected before any device work.
    for kw, code in [(dict(dt=1.0), P.PIC_E_CFL), (dict(dt=0.9, ck_beta_x=0.3), P.PIC_E_ARG),
                     (dict(dt=0.9, ck_beta_z=-0.01), P.PIC_E_ARG),
                     (dict(dt=0.5, ndim=3, nx=8, ny=8, nz=8), P.PIC_E_ARG),
                     (dict(dt=0.75, ck_beta_x=0.0, ck_beta_z=0.0), P.PIC_E_CFL),  # beta = 0 is Yee
                     (dict(dt=0.9, field_solver=2), P.PIC_E_ARG)]:
        kw.setdefault("field_solver", P.PIC_CK)
        with pytest.raises(P.PicError) as e:
            P.pic_create(P.pic_config_default(**kw))
        assert e.value.code == code, kw
    # a stable CK configuration passes validation (and then needs a GPU)
    try:
        P.pic_destroy(P.pic_create(P.pic_config_default(field_solver=P.PIC_CK, dt=0.99)))
    except P.PicError as e:
        assert e.code == P.PIC_E_CUDA


def test_config_struct_layout_matches_header(tmp_path):
    # the ctypes mirror of pic_config has the C compiler's size and field offsets
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = [f[0] for f in P.pic_config._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", offsetof(pic_config, {n}));\n' for n in names)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "pic.h"\nint main(void) {\n'
                   '  printf("%zu\\n", sizeof(pic_config));\n' + body + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    inc = Path(__file__).resolve().parents[1] / "include"
    subprocess.run([cc, "-I", str(inc), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(P.pic_config)
    assert out[1:] == [getattr(P.pic_config, n).offset for n in names]


def test_destroy_null_is_noop():
    P.lib().pic_destroy(None)


def test_null_handles_are_rejected_without_a_gpu():
    import ctypes
    out = (ctypes.c_double * 3)()
    assert P.lib().pic_charge_residual(None, out) == P.PIC_E_ARG
    assert P.lib().pic_step(None, 1) == P.PIC_E_ARG
    w = ctypes.c_double()
    assert P.lib().pic_adjoint_forward(None, 10, 5, ctypes.byref(w)) == P.PIC_E_ARG


def test_breakdown_windows_agree_with_oracle():
    # The (4,4) interpolation of the Galerkin multiplier has a pole inside [0, 1] in narrow alpha
    # windows (the counterpart of the window Sec. 3 excises), below Yee's 2D limit and, reachable with
    # the CK solver, near 0.77-0.78. The library and the oracle, with different solvers, must refuse
    # exactly the same alphas.
    alphas = np.linspace(0.60, 0.99, 781)
    lib_bad, orc_bad = [], []
    for a in alphas:
        try:
            P.pic_compute_correction_coeffs(0, a)
        except P.PicError as e:
            assert e.code == P.PIC_E_SINGULAR
            lib_bad.append(a)
        if O.rational_coeffs(0, a)[0] != 0:
            orc_bad.append(a)
    assert lib_bad == orc_bad
    low = [a for a in lib_bad if a < 0.71]
    high = [a for a in lib_bad if a >= 0.71]
    assert 5 <= len(low) < 60 and min(low) > 0.64 and max(low) < 0.70
    assert 5 <= len(high) < 40 and min(high) > 0.765 and max(high) < 0.79


def test_binding_refuses_arrays_the_library_would_overrun():
    # the library reads np (= len(cell)) elements of every particle array and n samples of t and w
    n = 5
    part = {"cell": np.zeros(n, np.int32), "species": np.zeros(n, np.int32), "ox": np.zeros(n, np.float32),
            "oz": np.zeros(n, np.float32), "dux": np.zeros(n, np.float32), "duy": np.zeros(n, np.float32),
            "duz": np.zeros(n, np.float32)}
    assert P.make_state(P.PIC_HOST, None, part).np == n
    with pytest.raises(ValueError):
        P.make_state(P.PIC_HOST, None, dict(part, oz=np.zeros(n - 1, np.float32)))
    with pytest.raises(ValueError):
        P.make_state(P.PIC_HOST, None, dict(part, cell=np.zeros(n, np.int64)))
    torch = pytest.importorskip("torch")
    assert P.make_state(P.PIC_HOST, None, {k: torch.from_numpy(v) for k, v in part.items()}).np == n
    with pytest.raises(ValueError):
        P.pic_fit_growth_rate(np.arange(10.0), np.ones(9))
