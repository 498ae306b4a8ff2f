"""Compiled-netlist blobs (host only): save/load round trips, and every kind of damage the
loader must turn into DP_EPARSE before anything reaches a device - sizes, level bounds,
fanin ids at or above the cell's level, the fanout CSR and edge positions, the user-order
permutations, caps, bytecode ranges - plus a fuzz of single-byte flips."""
import struct

import numpy as np
import pytest

from paper_2608_03778_gb300 import dp, netgen
from tests._netlists import custom_case

ARRAYS = [("lvl_ptr", "i4"), ("fanin", "u4"), ("fout_ptr", "i4"), ("fout_edge", "i4"), ("edge_fpos", "i4"),
          ("net_of_user", "i4"), ("user_of_net", "i4"), ("cell_of_user", "i4"), ("user_of_cell", "i4"),
          ("base_cap", "f4"), ("pincap", "f4"), ("op_arity", "u1"), ("op_tt", "u2"), ("bc_ops", "u1"),
          ("bc_args", "i1"), ("bc_offset", "i4"), ("bc_length", "i4")]


def layout(blob):
    """Offsets of the blob's arrays (tag, six int64 sizes, then count + elements per array)."""
    assert blob[:8] == b"DPBLOB01"
    at = 8 + 6 * 8
    out = {}
    for name, dt in ARRAYS:
        n = struct.unpack_from("<q", blob, at)[0]
        at += 8
        out[name] = (at, n, np.dtype(dt))
        at += n * np.dtype(dt).itemsize
    assert at == len(blob)
    return out


def get(blob, lay, name):
    at, n, dt = lay[name]
    return np.frombuffer(blob, dt, n, at).copy()


def put(blob, lay, name, arr):
    at, n, dt = lay[name]
    b = bytearray(blob)
    b[at:at + n * dt.itemsize] = np.asarray(arr, dt).tobytes()
    return bytes(b)


def expect_parse_error(blob, what=""):
    with pytest.raises(dp.DPError) as e:
        c = dp.dp_compiled_load(blob)
        dp.dp_compiled_free(c)
    assert e.value.name == "DP_EPARSE"
    if what:
        assert what in str(e.value), str(e.value)


@pytest.fixture(scope="module")
def cases(library_text):
    rng = np.random.default_rng(3)
    out = [(netgen.netlist_text(netgen.WORKLOADS["small"]), library_text)]
    for _ in range(3):
        out.append(custom_case(rng, n_in=8, n_cells=60))
    return out


def test_round_trip(cases):
    for text, lib in cases:
        c = dp.dp_compile(text, lib)
        try:
            blob = dp.dp_compiled_save(c)
            c2 = dp.dp_compiled_load(blob)
            try:
                v1, v2 = dp.dp_compiled_view_get(c), dp.dp_compiled_view_get(c2)
                for k in v1:
                    if isinstance(v1[k], np.ndarray):
                        np.testing.assert_array_equal(v1[k], v2[k], err_msg=k)
                for f in ["n_nets", "n_start", "n_cells", "n_edges", "n_levels", "n_ops"]:
                    assert getattr(v1["info"], f) == getattr(v2["info"], f)
                assert dp.dp_compiled_save(c2) == blob
            finally:
                dp.dp_compiled_free(c2)
        finally:
            dp.dp_compiled_free(c)


@pytest.fixture(scope="module")
def blob(cases):
    text, lib = cases[1]
    c = dp.dp_compile(text, lib)
    b = dp.dp_compiled_save(c)
    dp.dp_compiled_free(c)
    return b


def test_sizes_and_framing(blob):
    expect_parse_error(b"", "not a blob")
    expect_parse_error(b"DPBLOB02" + blob[8:], "not a blob")
    expect_parse_error(blob[:-1], "sizes")
    expect_parse_error(blob + b"\0", "sizes")
    b = bytearray(blob)
    struct.pack_into("<q", b, 8, struct.unpack_from("<q", blob, 8)[0] + 1)   # n_nets off by one
    expect_parse_error(bytes(b))


def test_structural_damage(blob):
    lay = layout(blob)
    lvl = get(blob, lay, "lvl_ptr")
    fanin = get(blob, lay, "fanin")
    arity = get(blob, lay, "op_arity")
    ns = struct.unpack_from("<q", blob, 16)[0]
    # levels out of order
    bad = lvl.copy()
    bad[1], bad[2] = bad[2], bad[1]
    if bad[1] > bad[2]:
        expect_parse_error(put(blob, lay, "lvl_ptr", bad), "level bounds")
    # a first-level cell reading a net of its own level (a cycle through the level order)
    c = int(lvl[0])
    k = int(arity[fanin[4 * c] >> 24])
    assert k > 0
    bad = fanin.copy()
    own = ns + c   # the cell's own net
    bad[4 * c] = (bad[4 * c] & 0xFF000000) | own
    expect_parse_error(put(blob, lay, "fanin", bad))
    # a fanin id past the last net
    bad = fanin.copy()
    bad[4 * c] = (bad[4 * c] & 0xFF000000) | 0xFFFFF0
    expect_parse_error(put(blob, lay, "fanin", bad))
    # fanout edge pointing at an unused slot, and a wrong edge position
    fe = get(blob, lay, "fout_edge")
    bad = fe.copy()
    bad[0] = 4 * int(lvl[-1])   # a cell index past the last cell
    expect_parse_error(put(blob, lay, "fout_edge", bad), "fanout edge")
    ep = get(blob, lay, "edge_fpos")
    used = np.flatnonzero(ep >= 0)
    bad = ep.copy()
    bad[used[0]], bad[used[1]] = bad[used[1]], bad[used[0]]
    expect_parse_error(put(blob, lay, "edge_fpos", bad), "edge position")
    # user order not a permutation, or not the inverse of the other
    nou = get(blob, lay, "net_of_user")
    bad = nou.copy()
    bad[0] = bad[1]
    expect_parse_error(put(blob, lay, "net_of_user", bad), "user order")
    bad = nou.copy()
    bad[0], bad[1] = bad[1], bad[0]
    expect_parse_error(put(blob, lay, "net_of_user", bad), "user order")
    # caps: negative, NaN, infinite
    for v in [-1.0, np.nan, np.inf]:
        bad = get(blob, lay, "pincap")
        bad[0] = v
        expect_parse_error(put(blob, lay, "pincap", bad), "caps")
    # an arity above four
    bad = arity.copy()
    bad[fanin[4 * c] >> 24] = 5
    expect_parse_error(put(blob, lay, "op_arity", bad))
    # bytecode range past the end
    off = get(blob, lay, "bc_offset")
    bad = off.copy()
    bad[255] = 1 << 30
    expect_parse_error(put(blob, lay, "bc_offset", bad), "bytecode ranges")


def test_single_byte_flips_never_crash(blob):
    """Every flip either loads a structurally valid netlist or is rejected with DP_EPARSE."""
    rng = np.random.default_rng(11)
    for pos in rng.integers(0, len(blob), 300):
        b = bytearray(blob)
        b[int(pos)] ^= 1 << int(rng.integers(8))
        try:
            c = dp.dp_compiled_load(bytes(b))
        except dp.DPError as e:
            assert e.name in ("DP_EPARSE", "DP_ENOMEM"), e.name
            continue
        info = dp.dp_compiled_info(c)
        assert info.n_nets == info.n_start + info.n_cells
        dp.dp_compiled_free(c)
