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
    assert lib.pfem_abi_version() == 1
    assert lib.pfem_status_string(4) == b"capacity exceeded"
    assert lib.pfem_default_bins(1025, 2048 * 2048) == 1024
    assert lib.pfem_default_bins(33, 4096) == 32
    assert lib.pfem_default_bins(9, 10) == 8
    ws = lib.pfem_workspace_size(1025, 1024, 2048 * 2048, 4)
    assert ws >= 256 + 4 * (1024 * 1024 + 1) + 8 * 2048 * 2048


def test_bad_arguments_are_rejected_on_host(lib):
    null = ctypes.c_void_p(0)
    # n too small / C out of range / NULL buffers: PFEM_ERR_INVALID_ARG, nothing launched
    assert lib.pfem_interp_m2p(5, 10, null, 0, 1, null, null, 0, null) == 1
    assert lib.pfem_interp_m2p(33, 10, null, 0, 9, null, null, 0, null) == 1
    assert lib.pfem_project_p2m(33, 32, 4096, null, 0, null, null, null, 1, null, 0, 1, 0, null,
                                null, 0, 0, null, null, 0, null) == 1
    assert lib.pfem_build_cells(0, 10, null, 0, null, null, null, null, null, 0, null) == 1
    # workspace too small
    fake = ctypes.c_void_p(1 << 20)
    assert lib.pfem_build_cells(8, 100, fake, 0, fake, fake, fake, fake, fake, 16, null) == 3
    assert lib.pfem_read_status(null, None, None, null) == 1


def test_workspace_sizes_cover_queue_and_records(lib):
    """Quadratic P2M keeps an SVD-pass queue (8 bytes per node after byte 512) and 136 bytes of
    node record per node in the workspace; pfem_workspace_size covers both even when the
    binning scratch is small (few particles on a fine mesh).  The batched workspace covers the
    records plus an 8-byte node key per node when given the node total, and is the binning
    scratch alone without it."""
    n = 1025
    rec = 4 + 12 + 24 + 24 * 4
    assert lib.pfem_workspace_size(n, 32, 4096, 4) >= 512 + 8 * n * n + rec * n * n
    assert lib.pfem_workspace_size(n, 1024, 2048 * 2048, 4) >= 512 + 8 * n * n + rec * n * n
    nodes = 27_000_000
    assert lib.pfem_batch_workspace_size(10**6, 250_000, nodes) >= 256 + (rec + 8) * nodes
    bins_only = lib.pfem_batch_workspace_size(10**6, 250_000, 0)
    assert bins_only >= 4 * (250_000 + 1) + 8 * 10**6
    assert bins_only < 256 + (rec + 8) * nodes
    assert lib.pfem_batch_workspace_size(10**6, 250_000, -1) == 0
