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
    # og_config: 12 x uint32 + 2 x uint64; og_stats: 17 x uint64; og_query: 4 x uint32
    assert ctypes.sizeof(og.Config) == 64
    assert ctypes.sizeof(og.Stats) == 136
    assert ctypes.sizeof(og.Query) == 16


def _header():
    here = os.path.dirname(os.path.abspath(__file__))
    return open(os.path.join(here, "..", "include", "og.h")).read()


def test_constants_match_header_defines(og):
    """Every #define OG_<NAME> <number> of the header has the same value in the binding
    (OG_E_X -> E_X, OG_OK -> OK, OG_Q_X -> Q_X, OG_FUSION_OFF -> FUSION_OFF, ...)."""
    import re
    defs = dict(re.findall(r"^#define OG_([A-Z0-9_]+)\s+(0x[0-9A-Fa-f]+|[0-9]+)u?\b", _header(),
                           re.M))
    assert len(defs) >= 25
    for name, val in defs.items():
        assert hasattr(og, name), f"binding lacks {name}"
        assert getattr(og, name) == int(val, 0), name


def test_struct_fields_match_header(og):
    """The binding's Config / Stats / Query fields are the header's, in the same order."""
    import re
    text = _header()
    for cname, py in (("og_config", og.Config), ("og_stats", og.Stats), ("og_query", og.Query)):
        body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (cname, cname), text, re.S).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = re.findall(r"uint(32|64)_t\s+(\w+);", body)
        assert [n for _, n in fields] == [n for n, _ in py._fields_], cname
        for (bits, n), (pn, pt) in zip(fields, py._fields_):
            assert ctypes.sizeof(pt) * 8 == int(bits), (cname, n)


def test_library_does_not_link_the_oracle(og):
    data = open(og.LIB_PATH, "rb").read()
    assert b"or_dijkstra" not in data and b"liboracle" not in data


def test_null_arguments_are_rejected_before_any_device_call(og):
    """Entry points validate their arguments on the host first: a NULL graph or output, a
    bad mode or eps returns OG_E_INVALID without touching a GPU (none is present here)."""
    L = og.lib()
    out = (ctypes.c_uint32 * 4)()
    assert L.og_setcover(None, 10000, None, None, out, None, None) == og.E_INVALID
    assert L.og_kcore(None, 0, None, out, None, None) == og.E_INVALID
    fake = ctypes.c_void_p(1)  # never dereferenced: the bad eps / mode is checked first
    assert L.og_setcover(fake, 1000001, None, None, out, None, None) == og.E_INVALID
    assert L.og_setcover(fake, 10000, None, None, None, None, None) == og.E_INVALID
    assert L.og_kcore(fake, 7, None, out, None, None) == og.E_INVALID
    # vertex order: NULL graph, unknown order
    assert L.og_graph_set_order(None, og.ORDER_HOT_FIRST, None) == og.E_INVALID
    assert L.og_graph_set_order(fake, 3, None) == og.E_INVALID
    assert L.og_graph_get_order(None, None, None) == og.E_INVALID
    # probe: chain counts other than 1, 2, 4, 8, 16, threads not a multiple of 32, sizes
    # that are not powers of two, a footprint larger than the array
    ns = ctypes.c_double()
    for args in ((0, 1 << 20, 1 << 20, 4, 256, 3, 10), (0, 1 << 20, 1 << 20, 4, 256, 32, 10),
                 (0, 1 << 20, 1 << 20, 4, 100, 1, 10), (0, 3 << 20, 1 << 20, 4, 256, 1, 10),
                 (0, 1 << 20, 1 << 21, 4, 256, 1, 10), (3, 1 << 20, 1 << 20, 4, 256, 1, 10)):
        assert L.og_probe_chain(*args, ctypes.byref(ns)) == og.E_INVALID, args


def test_launch_status_mapping_on_hand_built_error_words(og):
    """Every round-engine entry point maps its launch's error word through one function
    (og_launch_status); its precedence is checked here on hand-built words."""
    T, A, S, B = 1, 2, 4, 8  # timeout, arena, saturation, failed bounds check
    assert og.launch_status(0) == og.OK
    assert og.launch_status(S) == og.E_OVERFLOW
    assert og.launch_status(T) == og.E_TIMEOUT
    assert og.launch_status(T | S) == og.E_TIMEOUT
    assert og.launch_status(0, arena_out=True) == og.E_ARENA
    assert og.launch_status(S, arena_out=True) == og.E_ARENA
    assert og.launch_status(T, arena_out=True) == og.E_TIMEOUT
    # the arena bit alone is not an error: the caller decides whether the arena can grow
    assert og.launch_status(A) == og.OK
    for extra in (0, T, A, S, T | A | S):
        assert og.launch_status(B | extra, 41, 7, 3, arena_out=bool(extra & A)) == og.E_INTERNAL
    assert og.launch_status(B, 41, 123, 5) == og.E_INTERNAL
    assert og.last_cuda_error() == "check 41 failed: value 123, context 5"
    assert og.launch_status(T) == og.E_TIMEOUT
    assert og.last_cuda_error() == "grid barrier wait gave up"
