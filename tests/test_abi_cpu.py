"""CPU-only checks of the C-ABI library: it builds, loads, exports every symbol the header
declares, and rejects bad host-side arguments without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pfem.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1610_05266_gb300 import build as B
    path = B.build()
    import paper_1610_05266_gb300._lib as L
    return L.load(path)


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(pfem_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_covers_header():
    import paper_1610_05266_gb300._lib as L
    assert set(declared_symbols()) <= set(L.SIGNATURES)


def test_host_queries(lib):
    assert lib.pfem_abi_version() == 2
    assert lib.pfem_status_string(4) == b"capacity exceeded"
    assert lib.pfem_default_bins(1025, 2048 * 2048) == 1024
    assert lib.pfem_default_bins(33, 4096) == 32
    assert lib.pfem_default_bins(9, 10) == 8
    ws = lib.pfem_workspace_size(1025, 1024, 2048 * 2048, 4)
    assert ws >= 256 + 4 * (1024 * 1024 + 1) + 8 * 2048 * 2048


def test_bad_arguments_are_rejected_on_host(lib):
    null = ctypes.c_void_p(0)
    # n too small / C out of range / NULL buffers: PFEM_ERR_INVALID_ARG, nothing launched
    assert lib.pfem_interp_m2p(null, 5, 10, null, 0, 1, null, null, 0, null) == 1
    assert b"out of range" in lib.pfem_last_error(null)
    assert lib.pfem_interp_m2p(null, 33, 10, null, 0, 9, null, null, 0, null) == 1
    assert lib.pfem_project_p2m(null, 33, 32, 4096, null, 0, null, null, null, 1, null, 0, 1, 0,
                                null, null, 0, 0, null, null, 0, null) == 1
    assert b"NULL" in lib.pfem_last_error(null)
    assert lib.pfem_build_cells(null, 0, 10, null, 0, null, null, null, null, null, 0, null) == 1
    # workspace too small
    fake = ctypes.c_void_p(1 << 20)
    assert lib.pfem_build_cells(null, 8, 100, fake, 0, fake, fake, fake, fake, fake, 16, null) == 3
    assert b"ws_bytes" in lib.pfem_last_error(null)
    assert lib.pfem_read_status(null, None, None, null) == 1


def test_context_options_and_last_error(lib):
    """pfem_create / pfem_get_options / pfem_last_error / pfem_destroy on the host: defaults are
    filled in, out-of-range options are refused with a message, and a context keeps the error
    text of the calls made with it (separately from calls without a context)."""
    import paper_1610_05266_gb300._lib as L
    d = L.Options()
    lib.pfem_options_default(ctypes.byref(d))
    assert (d.walk_max_steps, d.star_capacity, d.node_capacity, d.batch_tile_rows) == (64, 16, 24, 8)
    h = ctypes.c_void_p()
    bad = L.Options(star_capacity=2)
    assert lib.pfem_create(ctypes.byref(h), ctypes.byref(bad)) == 1
    assert not h.value and b"star_capacity" in lib.pfem_last_error(None)
    bad = L.Options(batch_tile_rows=5)
    assert lib.pfem_create(ctypes.byref(h), ctypes.byref(bad)) == 1
    opt = L.Options(walk_max_steps=-1, star_capacity=3, search_radius_max=2)
    assert lib.pfem_create(ctypes.byref(h), ctypes.byref(opt)) == 0 and h.value
    got = L.Options()
    assert lib.pfem_get_options(h, ctypes.byref(got)) == 0
    assert (got.walk_max_steps, got.star_capacity, got.node_capacity, got.search_radius_max) == (-1, 3, 24, 2)
    null = ctypes.c_void_p(0)
    assert lib.pfem_interp_m2p(h, 9, 10, null, 0, 0, null, null, 0, null) == 1
    assert b"C = 0" in lib.pfem_last_error(h)
    lib.pfem_interp_m2p(null, 9, 10, null, 0, 1, null, null, 5, null)
    assert b"C = 0" in lib.pfem_last_error(h)               # the context's text is its own
    lib.pfem_destroy(h)
    lib.pfem_destroy(null)


def test_options_struct_matches_the_header(lib):
    """pfem_options as the binding lays it out is the header's struct: 16 int32 fields
    (64 bytes), and pfem_options_default writes inside it (a canary after it stays intact)."""
    import paper_1610_05266_gb300._lib as L
    assert ctypes.sizeof(L.Options) == 64
    buf = (ctypes.c_uint8 * (ctypes.sizeof(L.Options) + 64))(*([0xA5] * (ctypes.sizeof(L.Options) + 64)))
    lib.pfem_options_default(ctypes.cast(buf, ctypes.c_void_p))
    assert all(b == 0xA5 for b in bytes(buf)[ctypes.sizeof(L.Options):])
    got = L.Options.from_buffer_copy(bytes(buf)[:ctypes.sizeof(L.Options)])
    assert (got.walk_max_steps, got.star_capacity, got.node_capacity) == (64, 16, 24)
    assert all(r == 0 for r in got.reserved)


def test_values_and_stage_events_need_a_context(lib):
    """pfem_set_values_event / pfem_set_stage_events belong to a context: without one they are
    refused with a message; with one, setting and clearing them succeeds on the host (nothing
    is launched until a P2M call)."""
    null = ctypes.c_void_p(0)
    assert lib.pfem_set_values_event(null, null) == 1
    assert b"needs a context" in lib.pfem_last_error(None)
    assert lib.pfem_set_stage_events(null, null, 0) == 1
    h = ctypes.c_void_p()
    assert lib.pfem_create(ctypes.byref(h), None) == 0
    assert lib.pfem_set_values_event(h, ctypes.c_void_p(0x1234)) == 0   # stored, not used here
    assert lib.pfem_set_values_event(h, null) == 0
    assert lib.pfem_set_stage_events(h, null, 9) == 1
    assert b"0..8" in lib.pfem_last_error(h)
    assert lib.pfem_set_stage_events(h, null, 0) == 0
    lib.pfem_destroy(h)


def test_python_context_wrapper():
    import paper_1610_05266_gb300 as P
    ctx = P.Context(walk_max_steps=3, star_capacity=5)
    o = ctx.options()
    assert o["walk_max_steps"] == 3 and o["star_capacity"] == 5 and o["node_capacity"] == 24
    with pytest.raises(P.PfemError) as e:
        P.Context(node_capacity=99)
    assert "node_capacity" in str(e.value)


def test_workspace_sizes_cover_queue_and_records(lib):
    """P2M keeps in the workspace a fix-pass queue (8 bytes per node after byte 512), 136 bytes
    of node record per node and the star table (64 + 8 bytes per particle); pfem_workspace_size
    covers them even when the binning scratch is small (few particles on a fine mesh).  The
    batched workspace covers the queue, the records plus an 8-byte node key per node and the
    star table when given the node total, and is the binning scratch alone without it."""
    n = 1025
    rec = 4 + 12 + 24 + 24 * 4
    tab = 64 + 8
    N = 2048 * 2048
    assert lib.pfem_workspace_size(n, 32, 4096, 4) >= 512 + 8 * n * n + rec * n * n + tab * 4096
    assert lib.pfem_workspace_size(n, 1024, N, 4) >= 512 + 8 * n * n + rec * n * n + tab * N
    nodes = 27_000_000
    assert lib.pfem_batch_workspace_size(10**6, 250_000, nodes) >= 256 + (8 + rec + 8) * nodes + tab * 10**6
    bins_only = lib.pfem_batch_workspace_size(10**6, 250_000, 0)
    assert bins_only >= 4 * (250_000 + 1) + 8 * 10**6
    assert bins_only < 256 + (rec + 8) * nodes
    assert lib.pfem_batch_workspace_size(10**6, 250_000, -1) == 0
