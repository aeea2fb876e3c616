"""Test helpers on gate lists (structure only)."""
import numpy as np


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
