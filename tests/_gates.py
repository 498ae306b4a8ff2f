"""Test-side ground truth for the 13 generator gates, written independently of
the oracle: Boolean lambdas on numpy arrays (any integer dtype, bitwise) and
closed-form SP / partial derivatives under input independence."""
import numpy as np

ALL = ~np.uint64(0)


def _n(x):
    return ~x if x.dtype == np.uint64 else 1 - x


# name -> (input pins, output pin, Boolean function on 0/1 ints or on uint64 words)
BOOL = {
    "INV": (["A"], "ZN", lambda a: _n(a)),
    "BUF": (["A"], "Z", lambda a: a),
    "NAND2": (["A1", "A2"], "ZN", lambda a, b: _n(a & b)),
    "NOR2": (["A1", "A2"], "ZN", lambda a, b: _n(a | b)),
    "AND2": (["A1", "A2"], "ZN", lambda a, b: a & b),
    "OR2": (["A1", "A2"], "ZN", lambda a, b: a | b),
    "XOR2": (["A", "B"], "Z", lambda a, b: a ^ b),
    "XNOR2": (["A", "B"], "ZN", lambda a, b: _n(a ^ b)),
    "NAND3": (["A1", "A2", "A3"], "ZN", lambda a, b, c: _n(a & b & c)),
    "NOR3": (["A1", "A2", "A3"], "ZN", lambda a, b, c: _n(a | b | c)),
    "AOI21": (["A1", "A2", "B"], "ZN", lambda a1, a2, b: _n((a1 & a2) | b)),
    "OAI21": (["A1", "A2", "B"], "ZN", lambda a1, a2, b: _n((a1 | a2) & b)),
    "MUX2": (["A", "B", "S"], "Z", lambda a, b, s: (a & _n(s)) | (b & s)),
}

# closed-form P(out = 1) for independent inputs with P(in_i = 1) = p_i
SP = {
    "INV": lambda a: 1 - a,
    "BUF": lambda a: a,
    "NAND2": lambda a, b: 1 - a * b,
    "NOR2": lambda a, b: (1 - a) * (1 - b),
    "AND2": lambda a, b: a * b,
    "OR2": lambda a, b: a + b - a * b,
    "XOR2": lambda a, b: a + b - 2 * a * b,
    "XNOR2": lambda a, b: 1 - a - b + 2 * a * b,
    "NAND3": lambda a, b, c: 1 - a * b * c,
    "NOR3": lambda a, b, c: (1 - a) * (1 - b) * (1 - c),
    "AOI21": lambda a1, a2, b: (1 - a1 * a2) * (1 - b),
    "OAI21": lambda a1, a2, b: 1 - (a1 + a2 - a1 * a2) * b,
    "MUX2": lambda a, b, s: a * (1 - s) + b * s,
}

# closed-form partial derivatives d SP / d p_i, one lambda per input
DSP = {
    "INV": [lambda a: -1.0],
    "BUF": [lambda a: 1.0],
    "NAND2": [lambda a, b: -b, lambda a, b: -a],
    "NOR2": [lambda a, b: -(1 - b), lambda a, b: -(1 - a)],
    "AND2": [lambda a, b: b, lambda a, b: a],
    "OR2": [lambda a, b: 1 - b, lambda a, b: 1 - a],
    "XOR2": [lambda a, b: 1 - 2 * b, lambda a, b: 1 - 2 * a],
    "XNOR2": [lambda a, b: 2 * b - 1, lambda a, b: 2 * a - 1],
    "NAND3": [lambda a, b, c: -b * c, lambda a, b, c: -a * c, lambda a, b, c: -a * b],
    "NOR3": [lambda a, b, c: -(1 - b) * (1 - c), lambda a, b, c: -(1 - a) * (1 - c),
             lambda a, b, c: -(1 - a) * (1 - b)],
    "AOI21": [lambda a1, a2, b: -a2 * (1 - b), lambda a1, a2, b: -a1 * (1 - b),
              lambda a1, a2, b: -(1 - a1 * a2)],
    "OAI21": [lambda a1, a2, b: -(1 - a2) * b, lambda a1, a2, b: -(1 - a1) * b,
              lambda a1, a2, b: -(a1 + a2 - a1 * a2)],
    "MUX2": [lambda a, b, s: 1 - s, lambda a, b, s: s, lambda a, b, s: b - a],
}

NAMES = list(BOOL)
PINCAP = {"X1": 0.8, "X2": 1.6, "X4": 3.2}


def parse_netlist(text):
    """Minimal independent reader of the netlist text: returns (nets{name: idx}, wire[],
    inputs[], dffs[(d, q)], cells[(ref, {pin: net})]) with net indices in declaration order."""
    nets, wire, inputs, dffs, cells = {}, [], [], [], []
    for line in text.splitlines():
        line = line.split("#", 1)[0].split()
        if not line:
            continue
        kw = line[0]
        if kw == "net":
            nets[line[1]] = len(wire)
            wire.append(float(line[2]))
        elif kw == "input":
            inputs.append(nets[line[1]])
        elif kw == "dff":
            pins = dict(t.split("=") for t in line[3:])
            dffs.append((nets[pins["D"]], nets[pins["Q"]]))
        elif kw == "cell":
            cells.append((line[2], {p: nets[n] for p, n in (t.split("=") for t in line[3:])}))
    return nets, wire, inputs, dffs, cells


def gate_of(ref):
    return ref.rsplit("_", 1)[0]


def boolean_eval(text, start_values):
    """Evaluates every net of a netlist from values at the startpoints (order of appearance).
    ``start_values`` is [n_start, ...] of 0/1 ints or uint64 words; returns [n_nets, ...]."""
    nets, wire, inputs, dffs, cells = parse_netlist(text)
    starts = inputs + [q for _, q in dffs]
    val = [None] * len(wire)
    for k, n in enumerate(starts):
        val[n] = start_values[k]
    pending = list(cells)
    while pending:
        rest = []
        for ref, pins in pending:
            ins, out, fn = BOOL[gate_of(ref)]
            args = [val[pins[p]] for p in ins]
            if any(a is None for a in args):
                rest.append((ref, pins))
                continue
            val[pins[out]] = fn(*args)
        if len(rest) == len(pending):
            raise ValueError("cycle")
        pending = rest
    return np.array(val)
