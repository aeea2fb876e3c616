import numpy as np

import oracle
from circuit_utils import inverse_circuit
from paper_2009_01845_gb300 import inputs as qi


def test_inverse_circuit_undoes_every_kind():
    n = 6
    gates = qi.random_mixed_circuit(n, 80, seed=3, max_controls=2, max_unitary_k=3)
    psi = qi.random_state(n, 2)
    back = oracle.apply_circuit(oracle.apply_circuit(psi.copy(), n, gates), n, inverse_circuit(gates))
    assert np.max(np.abs(back - psi)) < 1e-13
