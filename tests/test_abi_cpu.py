"""Host-side checks of the C ABI that need no GPU."""

import ctypes
import os
import re

import pytest

import paper_1008_2192_gb300._lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(crb_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = L.load()
    names = declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    assert set(declared_functions()) <= set(L.SIGNATURES)


@pytest.mark.parametrize("args", [
    (0.0, 5.0, 4.5, 0.5, 1.0, 4), (7.0, -1.0, 4.5, 0.5, 1.0, 4), (7.0, 5.0, 0.0, 0.5, 1.0, 4),
    (7.0, 5.0, 4.5, 0.0, 1.0, 4), (7.0, 5.0, 4.5, 0.5, 0.0, 4), (7.0, 5.0, 4.5, 0.5, 1.0, -1),
    (float("nan"), 5.0, 4.5, 0.5, 1.0, 4),
])
def test_create_rejects_invalid_parameters(args):
    lib = L.load()
    assert not lib.crb_create(*args)
    assert b"invalid parameters" in lib.crb_last_error()


def test_null_context_and_strerror():
    lib = L.load()
    assert lib.crb_clean(None, None, 1, 1, None, None, None) == L.CRB_EINVAL
    assert lib.crb_sync_status(None, None) == L.CRB_EINVAL
    assert lib.crb_strerror(L.CRB_EALIAS) == b"output overlaps input"
    assert lib.crb_strerror(99) == b"unknown status"
    tw, th = ctypes.c_int(), ctypes.c_int()
    shapes = []
    for i in range(lib.crb_num_tile_shapes()):
        assert lib.crb_tile_shape(i, ctypes.byref(tw), ctypes.byref(th)) == 0
        assert tw.value % 32 == 0 and th.value > 0
        shapes.append((tw.value, th.value))
    # index 0 is the default 64 x 32; index 5 the single-buffered 64 x 28 that tile_shape 0 takes when
    # its tiles fit one round of resident blocks and those of 64 x 32 do not
    assert shapes[0] == (64, 32) and shapes[5] == (64, 28)
    assert lib.crb_tile_shape(-1, None, None) == L.CRB_EINVAL
    assert lib.crb_tile_shape(len(shapes), None, None) == L.CRB_EINVAL


def test_networks_exhaustive_zero_one():
    """The selection networks (5 to 25 inputs) are correct on every 0/1 input (0-1 principle); the
    row-group network of four adjacent 5x5 medians on every 0/1 input with sorted columns, and its
    column sorter on every 0/1 input; all of them on random real inputs with ties."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "gen_networks", os.path.join(ROOT, "paper_1008_2192_gb300", "csrc", "gen_networks.py"))
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    for (_, n, rank) in g.SPECS:
        c, d, order, out = g.best_network(n, rank)
        g.verify(n, rank, d, order, out, exhaustive=True)
    for (_, groups) in g.ROW_SPECS:
        d, order, outs = g.row_network(groups)
        g.verify_row(groups, d, order, outs, exhaustive=True)


def test_row_network_mutants_are_caught():
    """The row-group checks catch a wrong root and an unsorted column: an output replaced by one operand
    of its last comparison, and a network whose columns skip their sort, both fail verify_row."""
    import importlib.util
    import pytest
    spec = importlib.util.spec_from_file_location(
        "gen_networks", os.path.join(ROOT, "paper_1008_2192_gb300", "csrc", "gen_networks.py"))
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    d, order, outs = g.row_network(4)
    # an output replaced by one operand of its last comparison
    k = d.defs[outs[1]]
    assert k[0] in ("min", "max")
    bad = list(outs)
    bad[1] = k[1]
    with pytest.raises(AssertionError):
        g.verify_row(4, d, g.live_order(d, bad), bad, exhaustive=False)
    # columns merged unsorted
    orig = g.sort_nodes
    try:
        g.sort_nodes = lambda dd, xs: list(xs) if len(xs) == g.ROW_D else orig(dd, xs)
        d2, order2, outs2 = g.row_network(4)
    finally:
        g.sort_nodes = orig
    with pytest.raises(AssertionError):
        g.verify_row(4, d2, order2, outs2, exhaustive=False)


def test_server_rejects_invalid_arguments():
    lib = L.load()
    opt = L.crb_options(0, 0, 0, 0, 0, 0)
    assert not lib.crb_server_create(7.0, 5.0, 4.5, 0.5, 1.0, 4, ctypes.byref(opt), 1 << 30, 0, 8)
    assert not lib.crb_server_create(7.0, 5.0, 4.5, 0.5, 1.0, 4, ctypes.byref(opt), 1 << 30, 2, 0)
    assert not lib.crb_server_create(7.0, 5.0, 4.5, 0.5, 1.0, 4, None, 0, 2, 8)
    assert lib.crb_server_submit(None, None, 1, 1, 7.0, 5.0, None, None, 0) == L.CRB_EINVAL
    assert lib.crb_server_poll(None, None, None, None, 0, 0) == -1


def test_binding_checks_outputs_before_the_call():
    """The C ABI cannot see how large a device buffer is, so the torch binding checks every output it
    passes (a contiguous CUDA tensor of the right dtype, shape and device) and the lengths of the
    per-frame arrays, raising before any library call."""
    torch = pytest.importorskip("torch")
    from paper_1008_2192_gb300 import api
    like = torch.zeros((3, 4))
    for bad in (torch.zeros((3, 4)), torch.zeros((4, 3)), torch.zeros((3, 4), dtype=torch.uint8), None):
        with pytest.raises(ValueError):
            api._check_out(bad, like, torch.float32, "out")  # host tensors are never valid outputs
    api._check_lengths(2, outs=[1, 2], masks=(3, 4), gains=None)
    with pytest.raises(ValueError, match="gains has 1 entries for 2 frames"):
        api._check_lengths(2, outs=[1, 2], gains=[7.0])
