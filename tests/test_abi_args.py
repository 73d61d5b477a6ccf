"""Argument checks of the device entry points run on the host before any
CUDA call, so they are tested here without a GPU: fake (never dereferenced)
device addresses, and calls that must be refused with MC_ERR_INVALID_ARG."""
import ctypes as C

from paper_2404_06359_gb300 import codec as mc

P = C.c_void_p
BAD = 1  # MC_ERR_INVALID_ARG


def _batch():
    b = mc.mc_device_batch()
    b.desc, b.payload, b.grids = 0x100000, 0x200000, 0x300000
    b.n_meshlets, b.n_grids, b.payload_bytes = 10, 1, 160
    b.total_tris, b.total_verts, b.max_block_words, b.max_tris = 100, 80, 32, 126
    return b


def test_cull_views_arguments_refused_on_the_host():
    lib, b = mc.lib(), _batch()
    vps, out, cnt, pos, st, scr = (P(0x400000), P(0x500000), P(0x600000), P(0x700000),
                                   P(0x800000), P(0x900000))
    call = lambda n, stride, v=vps, s=scr: lib.mc_decode_cull_views(C.byref(b), v, n, out, stride,
                                                                   cnt, pos, st, s, None, None)
    assert call(0, 300) == BAD        # no view
    assert call(9, 300) == BAD        # more than 8 views
    assert call(2, 299) == BAD        # region shorter than 3 * total_tris
    assert call(2, 300, v=P(0x400002)) == BAD   # matrices not 4-byte aligned
    assert call(2, 300, s=P(0x900004)) == BAD   # scratch not 16-byte aligned
    assert lib.mc_decode_cull_views(C.byref(b), vps, 2, out, 300, None, pos, st, scr, None,
                                    None) == BAD  # no counts
    g = P()
    assert lib.mc_graph_capture_cull_views(C.byref(b), vps, 0, out, 300, cnt, pos, st, scr, None,
                                           None, C.byref(g)) == BAD
    assert g.value is None


def test_batch_description_refused_on_the_host():
    lib, b = mc.lib(), _batch()
    args = (P(0x400000), P(0x500000), 300, P(0x600000), P(0x700000), P(0x800000), P(0x900000),
            None, None)
    for field, value in (("desc", 0x100008), ("n_grids", 0), ("max_block_words", 0),
                         ("payload_bytes", 161), ("n_attr", 6)):
        bb = _batch()
        setattr(bb, field, value)
        assert lib.mc_decode_cull_views(C.byref(bb), args[0], 2, args[1], args[2], args[3],
                                        args[4], args[5], args[6], None, None) == BAD, field


def test_ordered_cull_state_buffer_checked_on_the_host():
    lib, b = mc.lib(), _batch()
    assert lib.mc_cull_order_bytes(C.byref(b)) == 8 * 10 + 16
    assert lib.mc_decode_cull_ordered(C.byref(b), P(0x400000), P(0x500000), P(0x600000),
                                      P(0x700000), P(0x800000), P(0x900000), P(0xA00004), None,
                                      None) == BAD  # state words not 8-byte aligned
    assert lib.mc_decode_cull_ordered(C.byref(b), P(0x400000), P(0x500000), P(0x600000),
                                      P(0x700000), P(0x800000), P(0x900000), None, None,
                                      None) == BAD


def test_meshlet_count_limit_refused_on_the_host():
    """More than 2^31 meshlets is MC_ERR_LIMIT (2) from the batch decoders and the culls."""
    lib = mc.lib()
    bb = _batch()
    bb.n_meshlets = (1 << 31) + 1
    out = (P(0x400000), P(0x500000), P(0x600000), P(0x700000), P(0x800000))
    assert lib.mc_decode_batch(C.byref(bb), *out, None, None) == 2
    assert lib.mc_decode_cull_views(C.byref(bb), P(0x400000), 2, P(0x500000), 300, P(0x600000),
                                    P(0x700000), P(0x800000), P(0x900000), None, None) == 2
    bb.n_meshlets = 1 << 31  # the bound itself passes the count check (then fails on alignment)
    assert lib.mc_decode_batch(C.byref(bb), P(0x400000), P(0x500000), P(0x600000), P(0x700000),
                               P(0x800004), None, None) == BAD
