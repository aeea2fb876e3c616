"""Test helpers on gate lists (structure only)."""
import numpy as np

from paper_2009_01845_gb300 import inputs as qi


def inverse_circuit(gates):
    """The inverse queue: reversed order, each gate replaced by its inverse
    (U3(t, p, l)^-1 = U3(-t, -l, -p); U2(p, l) = U3(pi/2, p, l); rotations
    and phases negate their angle; S <-> SDG, T <-> TDG; UNITARY -> conjugate
    transpose; self-inverse gates unchanged)."""
    inv = {"S": "SDG", "SDG": "S", "T": "TDG", "TDG": "T"}
    out = []
    for g in reversed(gates):
        if g.kind == "U3":
            th, ph, la = g.params
            out.append(g._replace(params=(-th, -la, -ph)))
        elif g.kind == "U2":
            ph, la = g.params
            out.append(g._replace(kind="U3", params=(-np.pi / 2, -la, -ph)))
        elif g.kind in ("RX", "RY", "RZ", "U1", "CU1"):
            out.append(g._replace(params=(-g.params[0],)))
        elif g.kind in inv:
            out.append(g._replace(kind=inv[g.kind]))
        elif g.kind == "UNITARY":
            out.append(g._replace(matrix=np.conj(np.asarray(g.matrix)).T))
        else:
            out.append(g)
    return out


def near_swap_circuit(n, layers, seed):
    """U3 gates whose rotation is closer to a swap than to the identity
    (theta in (pi/2, pi)), with CZ, controlled-CZ and CU1 on the same qubits,
    an X and a controlled RZ per layer: in the tiled pass the swaps stay in
    the register frame, which the later sign flips, diagonal blocks and
    rotations of the stage must be written for."""
    r = qi.rng(seed)
    gates = []
    for l in range(layers):
        for q in range(n):
            th = float(r.uniform(2.0, 3.1))
            gates.append(qi.Gate("U3", (q,), (), (th, float(r.uniform(0, 6.28)), float(r.uniform(0, 6.28)))))
        for q in range(l % 3, n - 2, 3):
            gates.append(qi.Gate("CZ", (q, q + 1), (q + 2,)))
            gates.append(qi.Gate("CZ", (q + 1, q + 2)))
            gates.append(qi.Gate("CU1", (q, q + 2), (), (float(r.uniform(0, 6.28)),)))
        gates.append(qi.Gate("X", (l % n,)))
        gates.append(qi.Gate("RZ", ((l + 4) % n,), ((l + 1) % n,), (float(r.uniform(0, 6.28)),)))
    return gates
