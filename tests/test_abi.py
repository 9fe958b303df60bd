"""The C-ABI library builds, loads without a GPU, exports every symbol include/lfsgm.h
declares, and its Python mirror of lfsgm_config has the C layout.  Config validation is
host logic that runs before any CUDA call, so it is checked here on the CPU."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lfsgm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1907_13449_gb300 import _build
    _build.build()
    import paper_1907_13449_gb300 as lf
    return lf.load()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lfsgm_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_stage_entry_points():
    names = declared_functions()
    for n in ["lfsgm_create", "lfsgm_initial_disparity", "lfsgm_cost_volume", "lfsgm_sgm_aggregate",
              "lfsgm_wta_subpixel", "lfsgm_backward", "lfsgm_sync", "lfsgm_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_covers_every_declared_symbol():
    import paper_1907_13449_gb300 as lf
    for n in declared_functions():
        assert callable(getattr(lf, n, None)), n


def test_config_layout_matches_header():
    import paper_1907_13449_gb300 as lf
    fields = [f for f, _ in lf.Config._fields_]
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"lfsgm.h\"\nint main(void){\n"
    src += 'printf("%zu\\n", sizeof(lfsgm_config));\n'
    for f in fields:
        src += f'printf("%zu\\n", offsetof(lfsgm_config, {f}));\n'
    src += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = [int(x) for x in subprocess.check_output([exe]).split()]
    assert out[0] == C.sizeof(lf.Config)
    for f, off in zip(fields, out[1:]):
        assert getattr(lf.Config, f).offset == off, f


def _raw_create(lib, **kw):
    import lfsynth
    import paper_1907_13449_gb300 as lf
    p = lfsynth.tiny_params()
    cfg = lf.make_config(p)
    for k, v in kw.items():
        setattr(cfg, k, v)
    h = C.c_void_p()
    st = lib.lfsgm_create(C.byref(cfg), None, C.byref(h))
    return st, lib.lfsgm_last_error(None).decode()


@pytest.mark.parametrize("field,value,needle", [
    ("census_w", 6, "census_w"),
    ("dmax", -3.0, "dmin < dmax"),
    ("coarse_labels", 1, "coarse_labels"),
    ("coarse_labels", 300, "coarse_labels"),
    ("fine_labels", 1, "fine_labels"),
    ("fine_radius", -1, "fine_radius"),
    ("phi", 0.0, "phi"),
    ("fill_passes", 9, "fill_passes"),
    ("w_l2", -1.0, "weights"),
    ("p2_frac", 0.01, "p1_frac"),
    ("subpixel", 3, "subpixel"),
    ("softmin_tau", 0.0, "softmin_tau"),
    ("paths", 12, "paths"),
    ("edge_threshold", -1.0, "edge_threshold"),
    ("channels", 2, "channels"),
    ("boundless", 2, "boundless"),
    ("U", 1, None),
])
def test_invalid_config_rejected_before_any_cuda_call(lib, field, value, needle):
    kw = {field: value}
    if field == "U":
        kw["V"] = 1
        needle = "at least 2 views"
    st, msg = _raw_create(lib, **kw)
    assert st == 1, (st, msg)
    assert needle in msg


def test_null_arguments_rejected(lib):
    assert lib.lfsgm_create(None, None, None) == 1
    assert lib.lfsgm_destroy(None) == 1
    assert lib.lfsgm_sync(None) == 1
    assert lib.lfsgm_launch_count(None) == -1


def _cuda_present():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_cuda_present(), reason="placeholder pointers are only passed where no GPU can be reached")
def test_noalloc_rejects_a_misaligned_cost_before_any_cuda_call(lib):
    """Windowed rows are written as 16-byte vectors, so the allocation-free entry point refuses a
    cost buffer off a 16-byte boundary before it touches CUDA (INVALID_ARG = 1; with the check
    missing it would reach the CUDA runtime and fail differently)."""
    import lfsynth
    import paper_1907_13449_gb300 as lf
    cfg = lf.make_config(lfsynth.tiny_params())
    ptr = [C.c_void_p(v) for v in (256, 512, 768, 1024)]
    assert lib.lfsgm_cost_volume_noalloc(C.byref(cfg), None, *ptr, C.c_void_p(4096 + 4)) == 1
    assert lib.lfsgm_cost_volume_noalloc(C.byref(cfg), None, *ptr, C.c_void_p(4096 + 8)) == 1


def test_batch_arguments_rejected_before_any_cuda_call(lib):
    import lfsynth
    import paper_1907_13449_gb300 as lf
    out = C.c_void_p(123)
    assert lib.lfsgm_batch_create(0, None, None, None, None, 0, C.byref(out)) == 1
    assert out.value is None
    assert lib.lfsgm_batch_run(None) == 1
    assert lib.lfsgm_batch_destroy(None) == 1
    assert lib.lfsgm_batch_kernel_nodes(None) == -1
    cfgs = (lf.Config * 2)(lf.make_config(lfsynth.tiny_params(fine_labels=1)),
                           lf.make_config(lfsynth.tiny_params()))
    ptrs = (C.c_void_p * 2)(16, 32)          # never dereferenced: validation fails first
    assert lib.lfsgm_batch_create(2, cfgs, ptrs, ptrs, None, 0, C.byref(out)) == 1
    msg = lib.lfsgm_batch_last_error(None).decode()
    assert msg.startswith("light field 0") and "fine_labels" in msg


def test_batch_workspace_size_is_host_only(lib):
    """lfsgm_batch_workspace_size plans from the configurations alone (no GPU here): more
    branches need at least as much scratch, the autotuner's bound covers every candidate, and an
    invalid configuration is refused."""
    import lfsynth
    import paper_1907_13449_gb300 as lf
    params = [lfsynth.tiny_params(), lfsynth.bench_params(), lfsynth.tiny_params(census_w=7)]
    one = lf.lfsgm_batch_workspace_size(params, branches=1)
    two = lf.lfsgm_batch_workspace_size(params, branches=2)
    three = lf.lfsgm_batch_workspace_size(params, branches=3)
    auto = lf.lfsgm_batch_workspace_size(params, branches=0)
    assert 0 < one <= two <= three and auto >= max(one, two)
    assert one % 256 == 0
    with pytest.raises(lf.LfsgmError):
        lf.lfsgm_batch_workspace_size([lfsynth.tiny_params(census_w=9)], branches=1)
