"""Reader for the hand-worked fixtures in this folder."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    """Returns (library_text, netlist_text, values{key: [float]})."""
    sect, parts = None, {"library": [], "netlist": [], "values": []}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            s = line.strip()
            if not s or s.startswith("#"):
                continue
            if s.startswith("[") and s.endswith("]"):
                sect = s[1:-1]
                continue
            parts[sect].append(s)
    values = {}
    for s in parts["values"]:
        k, *v = s.split()
        values[k] = [float(x) for x in v]
    return "\n".join(parts["library"]) + "\n", "\n".join(parts["netlist"]) + "\n", values
