"""Plans: gate queues captured in CUDA graphs, strategy chosen by the
autotuner, replayed on the state's stream."""
import numpy as np
import pytest

import oracle
from paper_2009_01845_gb300 import inputs as qi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    from paper_2009_01845_gb300 import qsim
    qsim.load(build_if_missing=True)
    return qsim


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_autotuned_plan_replays_the_circuit(qs, dtype):
    n = 16
    gates = qi.random_layer_circuit(n, layers=6, seed=12)
    st = qs.State(n, dtype=dtype).init_basis(0)
    plan = qs.Plan(st, gates, mode="auto", autotune=True)
    info = plan.info()
    assert info["graph_nodes"] > 0
    assert info["mode"] in ("tiled", "fused", "unfused")
    assert info["schedule"] in ((0, 0), (1, 0), (2, 0), (0, 32))
    st.init_basis(0)
    plan.execute()
    plan.execute()               # the circuit twice
    want = oracle.run_circuit(n, gates + gates)
    tol = 1e-12 if dtype == "c128" else 1e-5
    assert np.max(np.abs(st.get() - want)) < tol


@pytest.mark.parametrize("mode", ["tiled", "fused", "unfused"])
def test_forced_mode_plans(qs, mode):
    n = 14
    gates = qi.random_mixed_circuit(n, 80, seed=33, max_controls=2, max_unitary_k=3)
    psi = qi.random_state(n, 4)
    st = qs.State(n, dtype="c64").set(psi)
    plan = qs.Plan(st, gates, mode=mode, autotune=False)
    assert plan.info()["mode"] == mode
    plan.execute()
    want = oracle.apply_circuit(psi.copy(), n, gates)
    assert np.max(np.abs(st.get() - want)) < 1e-5


def test_batched_plan_reads_current_parameters(qs):
    import torch
    n, B, L = 13, 3, 4
    th = qi.variational_params(B, L, n, seed=8)
    tmpl = qi.variational_circuit(n, th[0])
    pidx, P = qs.param_indices(tmpl)
    params = torch.tensor(th.reshape(B, -1), device="cuda")
    st = qs.State(n, batch=B, dtype="c128").init_basis(0)
    plan = qs.Plan(st, tmpl, mode="tiled", autotune=False, param_index=pidx, params=params)
    plan.execute()
    got = st.get()
    for b in range(B):
        assert np.max(np.abs(got[b] - oracle.run_circuit(n, qi.variational_circuit(n, th[b])))) < 1e-12
    params.mul_(0.5)             # new angles, same graph
    st.init_basis(0)
    plan.execute()
    got = st.get()
    for b in range(B):
        want = oracle.run_circuit(n, qi.variational_circuit(n, 0.5 * th[b]))
        assert np.max(np.abs(got[b] - want)) < 1e-12
