"""CPU-only checks of the library boundary: the shared library builds, loads
and exports every symbol include/treelik.h declares; the Python binding and
the op-list builders are consistent. No compute calls (no GPU here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_27607_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def header_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^int\s+(tl_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ("tl_create", "tl_destroy", "tl_set_tip_states", "tl_set_tip_partials",
                 "tl_set_pattern_weights", "tl_set_category_rates", "tl_set_category_weights",
                 "tl_set_model", "tl_set_eigen", "tl_update_matrices", "tl_update_partials",
                 "tl_root_loglik", "tl_update_pre_partials", "tl_pre_order_gradient",
                 "tl_edge_derivatives"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2606_27607_gb300 import _lib
    assert set(header_functions()) <= set(_lib.SIGNATURES)


def test_struct_layouts_match_header():
    from paper_2606_27607_gb300 import _lib
    assert _lib.OP_DTYPE.itemsize == 5 * 4
    assert _lib.PRE_OP_DTYPE.itemsize == 11 * 4
    assert _lib.EDGE_DTYPE.itemsize == 3 * 4
    assert _lib.ADJ_OP_DTYPE.itemsize == 8 * 4           # tl_adj_op: 8 ints
    assert _lib.EIG_OP_DTYPE.itemsize == 4 * 4 + 2 * 8   # tl_eig_op: 4 ints, 2 doubles
    assert _lib.EIG_OP_DTYPE.fields["len1"][1] == 16     # doubles 8-aligned after 4 ints


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """The numpy dtypes of the op structs against sizeof/offsetof from the
    host C compiler reading include/treelik.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2606_27607_gb300 import _lib
    src = tmp_path / "layout.c"
    src.write_text(
        "#include <stddef.h>\n#include <stdio.h>\n#include \"treelik.h\"\n"
        "int main(void) { printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(tl_op), sizeof(tl_pre_op),"
        " sizeof(tl_edge), sizeof(tl_adj_op), sizeof(tl_eig_op), offsetof(tl_eig_op, len1));"
        " return 0; }\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got == [_lib.OP_DTYPE.itemsize, _lib.PRE_OP_DTYPE.itemsize, _lib.EDGE_DTYPE.itemsize,
                   _lib.ADJ_OP_DTYPE.itemsize, _lib.EIG_OP_DTYPE.itemsize,
                   _lib.EIG_OP_DTYPE.fields["len1"][1]]


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2606_27607_gb300 import Instance, TreelikError
    with pytest.raises(TreelikError):
        Instance(4, 10, 4, 4, 6, 14, 1, "f32")


def test_op_lists_are_a_valid_traversal():
    import synth
    from paper_2606_27607_gb300 import tree
    t = synth.yule_tree(50, np.random.default_rng(0))
    post = tree.post_ops(t.children, 50)
    seen = set(range(50))
    for op in post:
        assert op["child1"] in seen and op["child2"] in seen
        seen.add(int(op["dest"]))
    assert int(post[-1]["dest"]) == 98
    pre = tree.pre_ops(t.children, 50, pre_base=49)
    assert pre[0]["parent_pre"] == -1
    produced = set()
    for op in pre:
        if op["parent_pre"] != -1:
            assert op["parent_pre"] in produced
        for c in range(2):
            if op["pre"][c] >= 0:
                produced.add(int(op["pre"][c]))
    edges = sorted(int(e) for op in pre for e in op["edge"])
    assert edges == list(range(98))


def test_tensor_core_category_limit_is_checked_before_any_device_call(lib):
    """The tensor-core kernels keep 2 x R x 64 accumulator columns in 512
    TMEM columns, so TF32 instances take at most four categories; the check
    runs before the device is touched (so it holds on a machine without one)."""
    import ctypes as C
    h = C.c_void_p()
    rc = lib.tl_create(8, 100, 61, 6, 14, 30, 1, 0x4, None, C.byref(h))
    assert rc == -8  # TL_ERR_UNSUPPORTED
    buf = C.create_string_buffer(256)
    lib.tl_last_error(None, buf, 256)
    assert b"at most 4 categories" in buf.value


def test_unbuilt_and_out_of_range_precisions_are_rejected_before_any_device_call(lib):
    """BF16X3 is reserved and not built; TF32 covers 5..64 states; FP32 is
    four-state only. Each is refused by tl_create before the device is
    touched."""
    import ctypes as C
    h = C.c_void_p()
    buf = C.create_string_buffer(256)
    for states, flags, text in ((61, 0x8, b"BF16X3"), (4, 0x4, b"5..64"), (20, 0x2, b"4 states")):
        rc = lib.tl_create(8, 100, states, 4, 14, 30, 1, flags, None, C.byref(h))
        assert rc == -8, (states, flags, rc)   # TL_ERR_UNSUPPORTED
        lib.tl_last_error(None, buf, 256)
        assert text in buf.value, buf.value


def test_ratio_transform_validates_on_the_host():
    """Malformed input is rejected before any device call."""
    from paper_2606_27607_gb300._lib import TreelikError, ratio_heights
    par = np.array([4, 4, 5, 5, 6, 6, -1])  # 4 tips: 0,1 -> 4; 2,3 -> 5; 4,5 -> root 6
    tip_h = np.zeros(4)
    rate = np.ones(7)
    with pytest.raises(TreelikError, match="TL_ERR_ARG"):
        ratio_heights(par, tip_h, [0.5, 1.5, 0.5], 2.0, rate)      # ratio outside (0, 1)
    with pytest.raises(TreelikError, match="TL_ERR_ARG"):
        ratio_heights(par, tip_h, [0.5, 0.5, 0.5], -1.0, rate)     # root below the tips
    bad = par.copy()
    bad[0] = 6
    with pytest.raises(TreelikError, match="TL_ERR_ARG"):
        ratio_heights(bad, tip_h, [0.5, 0.5, 0.5], 2.0, rate)      # root with three children


def test_autograd_refuses_parameter_gradients_it_cannot_give():
    """A model kind without parameter derivatives: the autograd Function
    says so before touching the device."""
    torch = pytest.importorskip("torch")
    from paper_2606_27607_gb300 import LogLikelihood
    t = torch.ones(5, dtype=torch.float64, requires_grad=True)
    th = torch.ones(16, dtype=torch.float64, requires_grad=True)
    with pytest.raises(ValueError, match="dlogL/dQ"):
        LogLikelihood.apply(t, th, None, "custom", np.full(4, 0.25))
