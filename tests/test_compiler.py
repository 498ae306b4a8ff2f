"""Host-side compiler and C-ABI surface (no GPU): Algorithm 1 bytecode, common-gate ids,
truth tables, levelization (Sec. III-A), renumbering, fanin records and the transposed
fanout CSR, and error reporting."""
import ctypes
import itertools
import os
import re

import numpy as np
import pytest

from tests import _gates as G
from tests._lib import ensure_built

ensure_built()
from paper_2608_03778_gb300 import dp, netgen  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "diffpower.h")).read()
    names = set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(dp_\w+)\s*\(", hdr, re.M))
    assert len(names) >= 20
    lib = ctypes.CDLL(dp.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(dp.EXPORTED) <= names


BC = {"IN": 0, "NOT": 1, "AND": 2, "OR": 3, "XOR": 4, "C0": 5, "C1": 6}


def test_bytecode_post_order():
    f = dp.dp_compile_function("!(A1 & A2)")
    assert f["ops"] == [BC["IN"], BC["IN"], BC["AND"], BC["NOT"]] and f["args"][:2] == [0, 1]
    f = dp.dp_compile_function("(A & !S) | (B & S)")
    # input order = first appearance: A, S, B
    assert f["n_inputs"] == 3
    assert f["ops"] == [0, 0, 1, 2, 0, 0, 2, 3] and f["args"] == [0, 1, 0, 0, 2, 1, 0, 0]
    assert dp.dp_compile_function("1")["ops"] == [BC["C1"]]


@pytest.mark.parametrize("expr,lid", [
    ("A", 0), ("!A", 1), ("A & B", 2), ("A | B", 3), ("!(A & B)", 4), ("!(A | B)", 5), ("A ^ B", 6),
    ("A & B & C", 7), ("!(A | B | C)", 10), ("A ^ B ^ C ^ D", 16), ("!(A ^ B)", -1), ("(A & B) | C", -1),
    ("A & (B & C)", -1), ("B & A", 2),
])
def test_common_gate_ids(expr, lid):
    assert dp.dp_compile_function(expr)["logic_id"] == lid


def run_bc(ops, args, bits):
    st = []
    for o, a in zip(ops, args):
        if o == 0: st.append(bits[a])
        elif o == 1: st.append(1 - st.pop())
        elif o in (2, 3, 4):
            b, x = st.pop(), st.pop()
            st.append(x & b if o == 2 else (x | b if o == 3 else x ^ b))
        else: st.append(o - 5)
    assert len(st) == 1
    return st[0]


@pytest.mark.parametrize("gate", G.NAMES)
def test_truth_tables_match_boolean_functions(gate, library_text):
    line = next(l for l in library_text.splitlines() if l.startswith(f"cell {gate}_X1 "))
    expr = line.split(None, 4)[4]
    f = dp.dp_compile_function(expr)
    ins, _, fn = G.BOOL[gate]
    order = []
    for tok in re.findall(r"[A-Za-z_]\w*", expr):
        if tok not in order:
            order.append(tok)
    for m in range(2 ** len(ins)):
        bits = [(m >> j) & 1 for j in range(len(order))]
        vals = {p: bits[j] for j, p in enumerate(order)}
        want = fn(*[np.int64(vals[p]) for p in ins])
        assert (f["tt"] >> m) & 1 == want
        assert run_bc(f["ops"], f["args"], bits) == want


@pytest.mark.parametrize("bad", ["A &", "(A | B", "A $ B", "", "A B"])
def test_bad_functions(bad):
    with pytest.raises(dp.DPError):
        dp.dp_compile_function(bad)


@pytest.fixture(scope="module")
def small_compiled(library_text):
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    c = dp.dp_compile(text, library_text)
    v = dp.dp_compiled_view_get(c)
    dp.dp_compiled_free(c)
    return text, v


def test_sizes_and_levels(small_compiled):
    text, v = small_compiled
    spec = netgen.WORKLOADS["small"]
    info = v["info"]
    assert (info.n_cells, info.n_start, info.n_nets, info.n_levels) == (spec.n_cells, spec.n_start,
                                                                        spec.n_cells + spec.n_start, spec.depth)
    ns, nc = info.n_start, info.n_cells
    fan = v["fanin"].reshape(nc, 4)
    op = fan[:, 0] >> 24
    nets = fan.copy()
    nets[:, 0] &= 0xFFFFFF
    ar = v["op_arity"][op]
    lvl = np.zeros(ns + nc, np.int64)
    lp = v["lvl_ptr"]
    assert lp[0] == 0 and lp[-1] == nc and (np.diff(lp) > 0).all()
    for l in range(1, info.n_levels + 1):
        lvl[ns + lp[l - 1]: ns + lp[l]] = l
    for c in range(nc):
        fl = [lvl[nets[c, j]] for j in range(ar[c])]
        assert lvl[ns + c] == 1 + max(fl, default=0)
        assert all(nets[c, j] == 0xFFFFFF for j in range(ar[c], 4))
    for l in range(1, info.n_levels + 1):
        assert (np.diff(op[lp[l - 1]: lp[l]].astype(int)) >= 0).all()


def test_fanout_is_transpose(small_compiled):
    text, v = small_compiled
    info = v["info"]
    nc = info.n_cells
    fan = v["fanin"].reshape(nc, 4)
    op = fan[:, 0] >> 24
    nets = fan.copy()
    nets[:, 0] &= 0xFFFFFF
    ar = v["op_arity"][op]
    edges = {}
    for c in range(nc):
        for j in range(ar[c]):
            edges.setdefault(int(nets[c, j]), []).append(4 * c + j)
    fp, fe = v["fout_ptr"], v["fout_edge"]
    assert fp[-1] == info.n_edges == int(ar.astype(np.int64).sum())
    for n in range(info.n_nets):
        got = list(fe[fp[n]: fp[n + 1]])
        assert got == sorted(edges.get(n, []))


def test_user_order_and_caps(small_compiled, library_text):
    text, v = small_compiled
    nets, wire, inputs, dffs, cells = G.parse_netlist(text)
    nou, cou = v["net_of_user"], v["cell_of_user"]
    info = v["info"]
    assert sorted(nou) == list(range(info.n_nets)) and sorted(cou) == list(range(info.n_cells))
    starts = inputs + [q for _, q in dffs]
    assert [nou[s] for s in starts] == list(range(info.n_start))
    dffcap = np.zeros(len(wire))
    for d, _ in dffs:
        dffcap[d] += 0.8
    np.testing.assert_allclose(v["base_cap"][nou], np.array(wire) + dffcap, rtol=1e-6)
    fan = v["fanin"].reshape(info.n_cells, 4)
    lib = {}
    for line in library_text.splitlines():
        if line.startswith("cell "):
            _, ref, out, cap, expr = line.split(None, 4)
            order = []
            for tok in re.findall(r"[A-Za-z_]\w*", expr):
                if tok not in order:
                    order.append(tok)
            lib[ref] = (out, float(cap), order)
    for u, (ref, pins) in enumerate(cells):
        out, cap, order = lib[ref]
        ic = cou[u]
        assert nou[pins[out]] == info.n_start + ic
        assert v["pincap"][ic] == np.float32(cap)
        for j, p in enumerate(order):
            assert (fan[ic, j] & (0xFFFFFF if j == 0 else 0xFFFFFFFF)) == nou[pins[p]]


def test_generated_ids_carry_bytecode(small_compiled):
    text, v = small_compiled
    for lid in range(32, 256):
        if v["bc_offset"][lid] < 0:
            continue
        o, n = v["bc_offset"][lid], v["bc_length"][lid]
        ops, args = v["bc_ops"][o:o + n], v["bc_args"][o:o + n]
        k = int(v["op_arity"][lid])
        for m in range(2 ** k):
            bits = [(m >> j) & 1 for j in range(k)]
            assert run_bc(list(ops), list(args), bits) == (int(v["op_tt"][lid]) >> m) & 1


@pytest.mark.parametrize("bad,code", [
    ("net a 1\nnet b 1\ninput a\ncell u INV_X1 A=b ZN=b\n", "DP_ECYCLE"),
    ("net a 1\nnet b 1\nnet c 1\ninput a\ncell u INV_X1 A=c ZN=b\ncell v INV_X1 A=b ZN=c\n", "DP_ECYCLE"),
    ("net a 1\nnet b 1\ninput a\n", "DP_EPARSE"),
    ("net a 1\nnet b 1\ninput a\ncell u NAND2_X1 A1=a ZN=b\n", "DP_EPARSE"),
    ("net a 1\nnet b 1\ninput a\ninput b\ncell u INV_X1 A=a ZN=b\n", "DP_EPARSE"),
    ("net a 1\nnet b 1\ninput a\ncell u NOPE A=a ZN=b\n", "DP_EPARSE"),
    ("net a x\n", "DP_EPARSE"),
    ("net a 1\nnet a 1\n", "DP_EPARSE"),
])
def test_malformed_netlists(bad, code, library_text):
    with pytest.raises(dp.DPError) as e:
        dp.dp_compile(bad, library_text)
    assert e.value.name == code


def test_wide_cells_unsupported():
    lib = "cell W5 Y 1.0 A & B & C & D & E\n"
    with pytest.raises(dp.DPError) as e:
        dp.dp_compile("net a 1\n", lib)
    assert e.value.name == "DP_EUNSUPPORTED"


def test_constant_cells_and_empty():
    lib = "cell TIEHI Y 1.0 1\ncell INV Y 1.0 !A\n"
    c = dp.dp_compile("net a 1\nnet y 1\ninput a\ncell t TIEHI Y=y\n", lib)
    v = dp.dp_compiled_view_get(c)
    dp.dp_compiled_free(c)
    assert v["info"].n_cells == 1 and v["info"].n_levels == 1 and v["info"].n_edges == 0
    c = dp.dp_compile("", lib)
    info = dp.dp_compiled_info(c)
    dp.dp_compiled_free(c)
    assert info.n_nets == 0 and info.n_cells == 0 and info.n_levels == 0


def test_abi_struct_layouts_match_the_header(tmp_path):
    """Every field offset and size of the C-ABI structs as the compiler lays them out,
    against the ctypes mirrors the binding passes."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc missing")
    structs = {"dp_config": dp.dp_config, "dp_info": dp.dp_info, "dp_server_config": dp.dp_server_config,
               "dp_request": dp.dp_request, "dp_server_stats": dp.dp_server_stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "diffpower.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        name, field, value = line.split()
        cls = structs[name]
        want = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert int(value) == want, (name, field)


def test_server_config_checked_before_any_device_call():
    """dp_server_create rejects a bad configuration with DP_EINVAL before it touches a device
    (so this runs without a GPU); the defaults are 64 requests per batch and one slot."""
    c = dp.server_config()
    assert c.max_batch == 64 and c.slots_per_design == 1 and c.plain == 0 and c.analysis.grad_mode == 0
    for bad in [dict(max_batch=0), dict(max_batch=4097), dict(slots_per_design=9), dict(slots_per_design=-1),
                dict(analysis=dp.config(grad_mode=1)), dict(analysis=dp.config(tr_mode=2))]:
        with pytest.raises(dp.DPError) as e:
            dp.dp_server_create(dp.server_config(**bad))
        assert e.value.name == "DP_EINVAL", bad
