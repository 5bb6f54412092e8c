"""The C ABI library loads and exports every entry point declared in include/og.h
(CPU only: no call here touches a GPU)."""
import ctypes
import os

import pytest


@pytest.fixture(scope="module")
def og():
    import paper_1911_07260_gb300 as og
    from paper_1911_07260_gb300 import build
    build.build()
    return og


def test_every_declared_symbol_is_exported(og):
    names = og.header_symbols()
    assert len(names) >= 20
    L = ctypes.CDLL(og.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert missing == []
    # and the binding declares a signature for each one
    for n in names:
        assert getattr(og.lib(), n).argtypes is not None, n


def test_error_strings_and_defaults(og):
    assert og.strerror(og.OK) == "ok"
    assert "timed out" in og.strerror(og.E_TIMEOUT)
    assert og.strerror(99) == "unknown error"
    c = og.Config()
    og.lib().og_config_default(ctypes.byref(c))
    assert c.fusion_threshold > 0 and c.expand_tile % 32 == 0 and c.spin_limit_ns > 0
    assert og.version() >= 100


def test_binding_fails_loudly_without_library(og, monkeypatch, tmp_path):
    monkeypatch.setattr(og, "_lib", None)
    monkeypatch.setattr(og, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        og.lib()


def test_structs_match_header(og):
    # og_config: 10 x uint32 + 2 x uint64; og_stats: 16 x uint64; og_query: 4 x uint32
    assert ctypes.sizeof(og.Config) == 64
    assert ctypes.sizeof(og.Stats) == 136
    assert ctypes.sizeof(og.Query) == 16


def test_library_does_not_link_the_oracle(og):
    data = open(og.LIB_PATH, "rb").read()
    assert b"or_dijkstra" not in data and b"liboracle" not in data
