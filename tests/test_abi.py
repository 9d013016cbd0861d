"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/amg_gb300.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_2511_21268_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "amg_gb300.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(amg_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("amg_opts_default", "amg_setup", "amg_pcg_solve", "amg_get_info", "amg_export_level",
                     "amg_free", "amg_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = _build.build_cuda()
    L = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(L, name), name
    L.amg_strerror.restype = ctypes.c_char_p
    assert L.amg_strerror(-5).startswith(b"matching")
    # argument checks run on the host, no device needed
    assert L.amg_opts_default(None) == -1
    assert L.amg_setup(None, None, None, None) == -1
    assert L.amg_mpnn_apply(None, None, 0) == -1
    assert L.amg_mpnn_loss_grad(None, None, 1, ctypes.c_uint64(0), None, None) == -1
    assert L.amg_mpnn_train(None, 1, None, 1, 1, ctypes.c_uint64(0), ctypes.c_float(0.01), None) == -1
    assert L.amg_div_check(ctypes.c_int64(-1), None, None, None, None, None) == -1
    assert L.amg_div_check(ctypes.c_int64(4), None, None, None, None, None) == -1
    assert L.amg_div_check(ctypes.c_int64(0), None, None, None, None, None) == 0


def test_binding_names_match_abi():
    from paper_2511_21268_gb300 import amg

    for name in declared_functions():
        assert hasattr(amg, name), name


def test_options_struct_defaults_through_the_binding_layout():
    """amg_opts_default (host only) fills the binding's struct: every field
    lands where the header puts it, the trailing network weights included."""
    from paper_2511_21268_gb300 import amg

    L = ctypes.CDLL(_build.build_cuda())
    o = amg.AmgOpts()
    assert L.amg_opts_default(ctypes.byref(o)) == 0
    assert (o.nu_pre, o.nu_post, o.match_passes, o.coarse_max, o.max_levels, o.dense_max) == (1, 1, 2, 200, 30, 4096)
    assert (o.testvec_sweeps, o.seed, o.stag, o.max_match_rounds) == (4, 20251126, 0.9, 1000)
    assert (o.precision, o.flexible, o.resid_replace_every, o.matrix_format) == (amg.AMG_FP64, 0, 20, 2)
    assert o.mpnn_weights is None and o.mpnn_bf16 == 1



def test_iga_size_closed_form_and_argument_checks():
    """amg_iga_size (host only): m^3 unknowns and the band's entry count
    (sum over rows of the per-direction band widths, cubed), and the
    argument checks of the assembly entry points."""
    from paper_2511_21268_gb300 import amg

    L = amg.lib()
    for n, p, wb in [(1, 1, 1), (1, 1, 0), (3, 2, 0), (7, 3, 1), (64, 3, 0), (96, 3, 1)]:
        P, _ = amg._iga_patch(n, p, with_boundary=wb)
        N, Z = amg.amg_iga_size(P)
        m = n + p if wb else n + p - 2
        T = sum(min(p, m - 1 - i) + min(p, i) + 1 for i in range(m))
        assert (N, Z) == (m ** 3, T ** 3)
    for bad in (dict(n=0, p=2), dict(n=4, p=0), dict(n=4, p=9), dict(n=4, p=2, nq=17), dict(n=300, p=2, nq=3),
                dict(n=4, p=2, geometry=7), dict(n=4, p=2, source=5)):
        P, _ = amg._iga_patch(**bad)
        try:
            amg.amg_iga_size(P)
            raise AssertionError(bad)
        except amg.AmgError as e:
            assert e.code == amg.AMG_ERR_ARG
    P, _ = amg._iga_patch(4, 2)
    P.kappa_m = 3  # features without their arrays
    assert L.amg_iga_size(ctypes.byref(P), ctypes.byref(ctypes.c_int64()), ctypes.byref(ctypes.c_int64())) == -1
    assert L.amg_iga_assemble(None, None, None, None, None, None, None) == -1
