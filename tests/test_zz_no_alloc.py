"""qaoa_energy_noalloc, the energy entry point that allocates no device
memory during the call (for callers that cannot allocate while they run),
against qaoa_energy on the same plan and parameters, two calls in a row.

This file is named to be collected last: a failure here leaves every other
test already run.
"""
import gc

import numpy as np
import pytest

from paper_2101_10296_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_REL_TOL = 1e-6
TERM_TOL = 1e-5


def _graphs():
    # register-resident cones (the 30-cycle) and large-state cones (C_30(1,2): 11
    # inner qubits, a random cubic graph on 16 vertices: 13, K_{8,8}: 16, six of
    # them outer qubits mixed in a shared-memory chunk pass)
    return [I.cycle(30), I.circulant(30, [1, 2]), I.random_regular(16, 3, 3), I.complete_bipartite(8, 8)]


def test_noalloc_energy_matches_qaoa_energy_twice(qlib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    graphs = _graphs()
    p = 3
    plan = qlib.Plan(graphs, p, orbits=False)
    plan.upload()
    assert plan.info()["n_big"] > 0
    n_reps = plan.info()["n_reps"]
    for call, seed in enumerate((3, 4)):
        theta = np.stack([I.draw_params(p, 12, seed + 10 * g) for g in range(len(graphs))])
        params = torch.tensor(theta, device="cuda")
        e_ref, t_ref = plan.energy(params, terms=True)
        out = torch.full((len(graphs), 12), float("nan"), dtype=torch.float64, device="cuda")
        terms = torch.full((n_reps, 12), float("nan"), dtype=torch.float64, device="cuda")
        plan.energy_noalloc(params, out=out, terms=terms)
        torch.cuda.synchronize()
        e_ref, t_ref = e_ref.cpu().numpy(), t_ref.cpu().numpy()
        e_na, t_na = out.cpu().numpy(), terms.cpu().numpy()
        assert np.all(np.isfinite(e_na)) and np.all(np.isfinite(t_na)), call
        assert np.allclose(e_na, e_ref, rtol=E_REL_TOL, atol=0), call
        assert np.max(np.abs(0.5 * (t_na - t_ref))) <= TERM_TOL, call
    assert plan.device_status() == 0


def test_noalloc_calls_leave_device_memory_unchanged(qlib):
    """After the plan's upload (set-up, which allocates), calls on register and
    large-state cones change neither the device's free memory nor torch's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    graphs = _graphs()
    p = 3
    plan = qlib.Plan(graphs, p, orbits=False)
    plan.upload()
    theta = np.stack([I.draw_params(p, 12, 7 + g) for g in range(len(graphs))])
    params = torch.tensor(theta, device="cuda")
    out = torch.empty(len(graphs), 12, dtype=torch.float64, device="cuda")
    gc.collect()  # plans of earlier tests free their device copies now, not during the calls
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    used0 = torch.cuda.memory_allocated()
    for _ in range(3):
        plan.energy_noalloc(params, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == used0
    assert plan.device_status() == 0


def test_noalloc_depth1_matches_and_allocates_nothing(qlib):
    """At p = 1 (a depth-1 plan: every cone's inner part is its edge) the
    allocation-free call takes the depth-1 kernel, like qaoa_energy: the same
    energies, and no device memory taken after the upload."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    graphs = [I.hypercube(7), I.torus(6, 6), I.cycle(30), I.random_regular(40, 3, 2)]
    plan = qlib.Plan(graphs, 1)
    plan.upload()
    assert plan.info()["depth1_kernel"] == 1
    theta = np.stack([I.draw_params(1, 20, 40 + g) for g in range(len(graphs))])
    params = torch.tensor(theta, device="cuda")
    e_ref = plan.energy(params).cpu().numpy()
    out = torch.full((len(graphs), 20), float("nan"), dtype=torch.float64, device="cuda")
    plan.energy_noalloc(params, out=out)
    gc.collect()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    used0 = torch.cuda.memory_allocated()
    plan.energy_noalloc(params, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == used0
    assert np.allclose(out.cpu().numpy(), e_ref, rtol=E_REL_TOL, atol=0)
    assert plan.device_status() == 0


def test_noalloc_rejects_bad_outputs_before_the_call(qlib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    plan = qlib.Plan(I.cycle(12), 2)
    plan.upload()
    params = torch.tensor(I.draw_params(2, 4, 0)[None], device="cuda")
    with pytest.raises(ValueError):
        plan.energy_noalloc(params, out=torch.empty(1, 4, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        plan.energy_noalloc(params, out=torch.empty(1, 3, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        plan.energy_noalloc(params, out=torch.empty(1, 8, dtype=torch.float64, device="cuda")[:, ::2])
    with pytest.raises(ValueError):
        plan.energy_noalloc(params, out=torch.empty(1, 4, dtype=torch.float64))
    assert plan.info()["n_reps"] == 1
    with pytest.raises(ValueError):
        plan.energy_noalloc(params, terms=torch.empty(2, 4, dtype=torch.float64, device="cuda"))


def test_noalloc_rejects_sizes_beyond_its_scratch(qlib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n, edges = I.hypercube(12)
    plan = qlib.Plan((n, edges), 1, full_cone=True)  # one 2^24-amplitude block: 128 MiB
    plan.upload()
    params = torch.tensor(I.draw_params(1, 2, 0)[None], device="cuda")
    with pytest.raises(qlib.QAOAError) as ei:
        plan.energy_noalloc(params)
    assert ei.value.code == qlib.QAOA_E_INVALID and "MiB" in str(ei.value)
