"""Host-side checks of the C ABI: the library loads, exports every declared symbol and
validates arguments before touching a device (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2506_18694_gb300 import hh

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hh.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"HH_API[^;]*?\b(hh_\w+)\s*\(", text, flags=re.S)))


def test_header_and_binding_agree():
    assert declared_symbols() == sorted(hh.EXPORTED)


def test_library_exports_every_declared_symbol(libhh):
    for name in declared_symbols():
        assert hasattr(libhh, name), name


def test_options_default(libhh):
    o = hh.default_options()
    assert (o.theta, o.levels, o.nu_pre, o.nu_post, o.nu_coarse) == (1.0, 4, 2, 2, 8)
    assert o.cycles_per_hss == 1 and o.omega == 0.0
    assert o.restart == 30 and o.precision == hh.HH_C64 and o.use_graphs == 1
    assert o.use_pdl == 1 and o.coarse_cluster_nodes == 100000 and o.tile_rows == 0 and o.autotune == 0
    assert o.fuse_sweeps == 1 and o.outer == hh.HH_OUTER_FGMRES and o.cycle_gamma == 1 and o.tile_form == 0 and o.smoother == hh.HH_SMOOTH_JACOBI


def test_footprint_bytes(libhh):
    o = hh.default_options()
    b2 = hh.footprint_bytes(2, 512, o)
    # Krylov basis alone: 61 complex128 vectors of 513^2 nodes
    assert b2 > 61 * 513 * 513 * 16
    assert hh.footprint_bytes(2, 1024, o) > 3.9 * b2
    assert hh.footprint_bytes(2, 100, o) == 0  # 100 is not divisible by 2^3
    assert hh.footprint_bytes(4, 64, o) == 0
    for bad in (dict(tile_form=3), dict(tile_form=-1), dict(tile_rows=3), dict(cycle_gamma=5), dict(smoother=2),
                dict(smoother=hh.HH_SMOOTH_GMRES, nu_coarse=9)):
        assert hh.footprint_bytes(2, 64, hh.default_options(**bad)) == 0, bad
    assert hh.footprint_bytes(2, 64, hh.default_options(tile_form=2)) == hh.footprint_bytes(2, 64, o)
    # mixed formulation: sigma entries n^d d 2^(d-1) in the Krylov vectors; one problem per object
    lib = hh.load_library()
    assert lib.hh_sigma_dofs(hh.Grid(2, 64)) == 64 * 64 * 4 and lib.hh_sigma_dofs(hh.Grid(3, 8)) == 8 ** 3 * 12
    mx = hh.default_options(formulation=hh.HH_FORM_MIXED)
    assert hh.footprint_bytes(2, 64, mx) - hh.footprint_bytes(2, 64, o) >= 61 * 64 * 64 * 4 * 16
    assert hh.footprint_bytes(2, 64, mx, nb=2) == 0
    assert hh.footprint_bytes(2, 64, hh.default_options(formulation=2)) == 0
    # GMRES smoother: max(nu) + 2 more level vectors per level (basis and work vector) and FP64 sums
    gm = hh.footprint_bytes(2, 64, hh.default_options(levels=2, smoother=hh.HH_SMOOTH_GMRES, nu_coarse=5))
    jac = hh.footprint_bytes(2, 64, hh.default_options(levels=2))
    assert gm - jac >= 7 * (65 * 65 + 33 * 33) * 8
    assert hh.footprint_bytes(2, 64, hh.default_options(levels=2, smoother=hh.HH_SMOOTH_GMRES, nu_coarse=8)) > gm


@pytest.mark.parametrize("dim,n,k,delta,dh,bc", [
    (4, 16, 10.0, 0.0, 2.0, [0] * 6),      # bad dimension
    (2, 12, 10.0, 0.0, 2.0, [0] * 4),      # 12 not divisible by 8
    (2, 16, -1.0, 0.0, 2.0, [0] * 4),      # k <= 0
    (2, 16, 10.0, -0.1, 2.0, [0] * 4),     # delta < 0
    (2, 16, 10.0, 0.0, 0.0, [0] * 4),      # delta_hat <= 0: H is not an inner product
    (2, 16, 10.0, 0.0, 2.0, [0, 2, 0, 0]),  # bad tag
])
def test_invalid_arguments_rejected_on_host(libhh, dim, n, k, delta, dh, bc):
    o = hh.default_options()
    arr = (ctypes.c_int * 6)(*(bc + [0] * (6 - len(bc))))
    out = ctypes.c_void_p(1234)
    st = libhh.hh_create_problem(ctypes.byref(hh.Grid(dim, n)), k, delta, dh, arr, ctypes.byref(o), None,
                                 ctypes.byref(out))
    assert st == -1 and not out.value
    assert libhh.hh_last_error()


def test_footprint_counts_w_cycle_buffers(libhh):
    v = hh.footprint_bytes(2, 256, hh.default_options(levels=4))
    w = hh.footprint_bytes(2, 256, hh.default_options(levels=4, cycle_gamma=2))
    # two complex64 vectors on each of levels 1..3
    assert w - v == 2 * 8 * (129 ** 2 + 65 ** 2 + 33 ** 2)


def test_footprint_is_linear_in_batch(libhh):
    # per problem the same bytes; per problem object 16 more (the persistent loop's barrier words)
    for dim, n in ((2, 256), (3, 32)):
        for prec in (hh.HH_C64, hh.HH_C128):
            o = hh.default_options(precision=prec)
            one = hh.footprint_bytes(dim, n, o) - 16
            assert one > 0 and hh.footprint_bytes(dim, n, o, nb=64) - 16 == 64 * one
    assert hh.footprint_bytes(2, 256, hh.default_options(), nb=0) == 0
    assert hh.footprint_bytes(3, 128, hh.default_options(), nb=600) == 0  # 129 * 600 > 65535


def _create_batch(libhh, dim, n, ks, ds, dhs, nb=None):
    o = hh.default_options()
    arr = (ctypes.c_int * 6)(*([0] * 6))
    D = ctypes.c_double * max(1, len(ks))
    out = ctypes.c_void_p(1234)
    st = libhh.hh_create_batch(ctypes.byref(hh.Grid(dim, n)), len(ks) if nb is None else nb, D(*ks), D(*ds), D(*dhs),
                               arr, ctypes.byref(o), None, ctypes.byref(out))
    return st, out


@pytest.mark.parametrize("dim,n,ks,ds,dhs,nb", [
    (2, 16, [10.0], [0.0], [2.0], 0),                       # empty batch
    (2, 16, [10.0, -3.0], [0.0, 0.0], [2.0, 2.0], None),    # one bad k
    (2, 16, [10.0, 5.0], [0.0, 0.0], [2.0, 0.0], None),     # one bad delta_hat
    (2, 16, [10.0, float("nan")], [0.0, 0.0], [2.0, 2.0], None),
    (3, 1024, [10.0] * 64, [0.0] * 64, [2.0] * 64, None),    # 1025 * 64 > 65535 launch planes
])
def test_invalid_batches_rejected_on_host(libhh, dim, n, ks, ds, dhs, nb):
    st, out = _create_batch(libhh, dim, n, ks, ds, dhs, nb)
    assert st == -1 and not out.value
    assert libhh.hh_last_error()


def test_status_strings(libhh):
    for s in (0, 1, -1, -2, -3, -4, -5):
        assert libhh.hh_status_string(s)


def test_server_validation_on_host(libhh):
    """Argument checks of the solve server that run before any device work."""
    o = hh.default_options()
    out = ctypes.c_void_p(1234)
    assert libhh.hh_server_create(0, 1 << 30, ctypes.byref(o), ctypes.byref(out)) == -1 and not out.value
    assert libhh.hh_server_create(2, 0, ctypes.byref(o), ctypes.byref(out)) == -1 and not out.value
    bad = hh.default_options(levels=20)
    assert libhh.hh_server_create(2, 1 << 30, ctypes.byref(bad), ctypes.byref(out)) == -1
    assert libhh.hh_last_error()
    mixed = hh.default_options(formulation=hh.HH_FORM_MIXED)
    assert libhh.hh_server_create(2, 1 << 30, ctypes.byref(mixed), ctypes.byref(out)) == -1 and not out.value


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the ABI structs have the C compiler's size and field offsets
    (a field added, dropped or reordered on one side only would corrupt every call)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"hh_grid": hh.Grid, "hh_options": hh.Options, "hh_info": hh.Info, "hh_request": hh.Request,
               "hh_server_stats": hh.ServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hh.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
