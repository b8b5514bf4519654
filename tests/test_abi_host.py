"""CPU checks of the C ABI: the library builds and loads, exports every entry
point declared in include/erem.h, and its host-side FP64 scalar routines
(Leja points, divided differences) agree with the oracle and with
high-precision arithmetic.  No CUDA computation runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import leja

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def E():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1209_5553_gb300 as E

    return E


def _declared_functions():
    src = ""
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src += open(os.path.join(ROOT, "include", f)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"EREM_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for want in ("erem_create", "erem_destroy", "pressure_solve", "erem_set_state", "phi1_apply",
                 "erem_step", "rosm_step", "erem_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(E):
    lib = ctypes.CDLL(E.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert set(_declared_functions()) == set(E.EXPORTED)


def test_struct_layouts_match_header(E):
    # sizes of the ABI structs as the C compiler lays them out
    assert ctypes.sizeof(E.erem_grid) == 4 * 4 + 3 * 8
    assert ctypes.sizeof(E.erem_physics) == 5 * 8 + 8
    assert ctypes.sizeof(E.erem_stats) % 8 == 0


def test_ensemble_struct_layouts_match_the_c_compiler(E, tmp_path):
    # the binding's ctypes layouts against the header as gcc lays it out
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "erem.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu %zu\\n", sizeof(erem_ens_config), '
                   'sizeof(erem_ens_member_stats), sizeof(erem_ens_run_stats), '
                   'offsetof(erem_ens_member_stats, alpha), offsetof(erem_ens_run_stats, cluster_ctas)); '
                   'return 0; }\n')
    exe = tmp_path / "sizes"
    import subprocess

    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == [ctypes.sizeof(E.erem_ens_config), ctypes.sizeof(E.erem_ens_member_stats),
                   ctypes.sizeof(E.erem_ens_run_stats), E.erem_ens_member_stats.alpha.offset,
                   E.erem_ens_run_stats.cluster_ctas.offset]


def test_krylov_struct_layouts_and_defaults(E, tmp_path):
    src = tmp_path / "kr.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "erem.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu\\n", sizeof(erem_krylov_opts), '
                   'sizeof(erem_krylov_stats), offsetof(erem_krylov_stats, deltas), '
                   'offsetof(erem_krylov_stats, t_ms)); return 0; }\n')
    exe = tmp_path / "kr"
    import subprocess

    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == [ctypes.sizeof(E.erem_krylov_opts), ctypes.sizeof(E.erem_krylov_stats),
                   E.erem_krylov_stats.deltas.offset, E.erem_krylov_stats.t_ms.offset]
    o = E.erem_krylov_opts()
    E.erem_default_krylov_opts(o)
    assert (o.tol_a, o.tol_r, o.m, o.max_substeps, o.n_replay) == (1e-6, 1e-6, 10, 1000, 0)


def test_stats_struct_layouts_match_the_c_compiler(E, tmp_path):
    src = tmp_path / "st.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "erem.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu %zu\\n", sizeof(erem_stats), '
                   'offsetof(erem_stats, degree_phi2), sizeof(erem_adapt_stats), '
                   'offsetof(erem_adapt_stats, t_reached), offsetof(erem_adapt_stats, t_ms)); '
                   'return 0; }\n')
    exe = tmp_path / "st"
    import subprocess

    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == [ctypes.sizeof(E.erem_stats), E.erem_stats.degree_phi2.offset,
                   ctypes.sizeof(E.erem_adapt_stats), E.erem_adapt_stats.t_reached.offset,
                   E.erem_adapt_stats.t_ms.offset]


def test_ensemble_create_rejects_bad_members_without_touching_the_gpu(E):
    ph = E.Physics().c()
    g2 = E.erem_grid(2, 8, 8, 1, 1.0, 1.0, 1.0)
    g3 = E.erem_grid(3, 8, 8, 8, 1.0, 1.0, 1.0)
    nonlinear = E.Physics(fluid_model=1).c()
    for grids, phys in [([g2, g3], [ph, ph]), ([g2], [nonlinear]), ([], [])]:
        with pytest.raises(E.EremError) as ei:
            E.erem_ensemble_create(grids, phys, E.EREM_FP32_BULK)
        assert ei.value.status == E.EREM_EINVAL
    assert E.erem_ensemble_last_error(None) != ""


def test_default_options(E):
    o = E.erem_leja_opts()
    E.erem_default_leja_opts(o)
    assert (o.tol_a, o.tol_r, o.p_order, o.m_max, o.max_doublings, o.avg_window) == \
        (1e-6, 1e-6, 2, 150, 6, 5)


def test_null_context_error_message(E):
    assert E.erem_last_error(None) != ""


def test_create_rejects_bad_grids_without_touching_the_gpu(E):
    # bad dimensions, empty extents, and grids whose padded cell count reaches
    # the 32-bit cell index (46344^2 in 2D, 1290^3 in 3D)
    for dims in [(4, 8, 8, 1), (2, 0, 8, 1), (2, 8, 8, 3), (3, 8, 8, 0), (2, 46344, 46344, 1),
                 (3, 1290, 1290, 1290)]:
        g = E.erem_grid(*dims, 1.0, 1.0, 1.0)
        with pytest.raises(E.EremError) as ei:
            E.erem_create(g, E.Physics().c(), E.EREM_FP64)
        assert ei.value.status == E.EREM_EINVAL


def test_host_leja_points_match_oracle(E):
    a = E.erem_leja_points(200)
    b = leja.leja_points(200)
    assert np.max(np.abs(a - b)) < 1e-14


@pytest.mark.parametrize("c,gamma", [(-20.0, 10.0), (-3.0, 1.5), (-60.0, 30.0), (-1e-6, 1e-8)])
def test_host_phi2_divided_differences_match_oracle(E, c, gamma):
    from oracle import nonauto

    xi = leja.leja_points(120)
    a = E.erem_phi2_divided_differences(xi, c, gamma)
    b = nonauto.phi2_divided_differences(xi, c, gamma)
    big = np.abs(b) > 1e-280
    assert np.max(np.abs(a[big] - b[big]) / np.abs(b[big])) < 1e-11


def test_host_fast_leja_points_match_oracle(E):
    # dyadic points: the library's incremental candidate update and the
    # oracle's fresh enumeration choose bit-identical points
    a = E.erem_fast_leja_points(300)
    b = leja.fast_leja_points(300)
    assert np.array_equal(a, b)
    with pytest.raises(ValueError):
        E.erem_fast_leja_points(5000)


@pytest.mark.parametrize("c,gamma", [(-20.0, 10.0), (-3.0, 1.5), (-60.0, 30.0), (-0.5, 0.25),
                                     (-200.0, 100.0), (-1e-6, 1e-8)])
def test_host_divided_differences_match_oracle(E, c, gamma):
    xi = leja.leja_points(150)
    a = E.erem_phi1_divided_differences(xi, c, gamma)
    b = leja.phi1_divided_differences(xi, c, gamma)
    m = np.abs(b) > 1e-280
    assert np.max(np.abs(a[m] - b[m]) / np.abs(b[m])) < 1e-12


def test_host_divided_differences_vs_high_precision(E):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 160
    xi = leja.leja_points(40)
    c, gamma = -12.5, 6.0
    d = E.erem_phi1_divided_differences(xi, c, gamma)
    xs = [mp.mpf(float(x)) for x in xi]
    col = [mp.expm1(mp.mpf(c) + gamma * x) / (mp.mpf(c) + gamma * x) for x in xs]
    ref = [col[0]]
    for j in range(1, len(xs)):
        col = [(col[i + 1] - col[i]) / (xs[i + j] - xs[i]) for i in range(len(col) - 1)]
        ref.append(col[0])
    for j, r in enumerate(ref):
        assert abs(d[j] - float(r)) <= 1e-11 * abs(float(r))
