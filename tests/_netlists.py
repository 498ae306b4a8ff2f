"""Small hand-built netlists shared by the CPU and GPU tests (text only, no arithmetic)."""

def custom_case(rng, n_in=6, n_cells=40, lib_extra=""):
    """Random reconvergent netlist over a library with 0..4-input cells (incl. constants,
    repeated pins in one expression and duplicated fanin nets)."""
    lib = ("cell AOI22 ZN 1.1 !((A1 & A2) | (B1 & B2))\n"
           "cell OAI211 ZN 0.9 !((A1 | A2) & B & C)\n"
           "cell MAJ Z 1.3 (A & B) | (A & C) | (B & C)\n"
           "cell XOR4 Z 2.0 A ^ B ^ C ^ D\n"
           "cell MUX2 Z 1.0 (A & !S) | (B & S)\n"
           "cell TIEHI Y 0.5 1\ncell TIELO Y 0.5 0\ncell BUF Z 0.7 A\ncell INV ZN 0.6 !A\n"
           "seq DFF D Q 0.8\n" + lib_extra)
    cells = [("AOI22", ["A1", "A2", "B1", "B2"], "ZN"), ("OAI211", ["A1", "A2", "B", "C"], "ZN"),
             ("MAJ", ["A", "B", "C"], "Z"), ("XOR4", ["A", "B", "C", "D"], "Z"), ("MUX2", ["A", "B", "S"], "Z"),
             ("TIEHI", [], "Y"), ("TIELO", [], "Y"), ("BUF", ["A"], "Z"), ("INV", ["A"], "ZN")]
    lines, avail = [], []
    for i in range(n_in + n_cells):
        lines.append(f"net n{i} {rng.uniform(0.5, 2.0):.5f}")
    for i in range(n_in - 2):
        lines.append(f"input n{i}")
        avail.append(i)
    lines.append(f"dff r0 DFF D=n{n_in + n_cells - 1} Q=n{n_in - 2}")
    lines.append(f"dff r1 DFF D=n{n_in + 3} Q=n{n_in - 1}")
    avail += [n_in - 2, n_in - 1]
    for c in range(n_cells):
        ref, pins, out = cells[rng.integers(len(cells))]
        ins = [avail[rng.integers(len(avail))] for _ in pins]   # duplicates allowed
        nid = n_in + c
        lines.append(f"cell u{c} {ref} " + " ".join(f"{p}=n{x}" for p, x in zip(pins, ins)) + f" {out}=n{nid}")
        avail.append(nid)
    return "\n".join(lines) + "\n", lib
