"""sph_diag_sums_noalloc: the conservation totals for callers that cannot
allocate device memory (a plug-in inside an application that owns all device
allocations).  It must agree with sph_diagnostics on the same state, call
after call, while keeping its partial sums in the library's fixed scratch
array instead of a caller workspace, take no device memory after its first
call, and agree with the CPU oracle's FP64 diagnostics of the same state.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_2405_03980_gb300 import _binding as B
from paper_2405_03980_gb300 import synth

pytestmark = pytest.mark.gpu

# FP64 sums over the same particles in a different order (input order here,
# cell order inside sph_diagnostics): the 1e-12 relative tolerance of the
# FP64 parity tests.
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _close(a, b, scale):
    return abs(a - b) <= TOL * max(abs(b), scale)


@pytest.mark.parametrize("precision", [B.SPH_FP64, B.SPH_MIXED])
def test_noalloc_sums_match_sph_diagnostics_twice(precision):
    import torch
    from paper_2405_03980_gb300.sim import Simulation

    c = synth.workload("cyl_8960", seed=2)
    sim = Simulation(c, precision=precision)
    sim.step(3)
    ref = sim.diagnostics()
    st = sim.state_arrays()
    dev = torch.device("cuda:0")
    pos = torch.from_numpy(st["pos"]).to(dev)
    vel = torch.from_numpy(st["vel"]).to(dev)
    spin = torch.from_numpy(st["spin"]).to(dev)
    rho = torch.from_numpy(st["rho"]).to(dev)
    sp = torch.from_numpy(c.species).to(dev)
    params = B.params_from_dict(c.params, precision=precision)
    outs = []
    dev_out = torch.full((B.SPH_DIAG_SUMS,), float("nan"), dtype=torch.float64, device=dev)
    # first call: host output (on a fresh device this call also loads the
    # module that holds the scratch array); second call: device output, which
    # must not take any device memory
    host_out = np.full(B.SPH_DIAG_SUMS, np.nan)
    B.sph_diag_sums_noalloc(params, c.n, pos, vel, spin, sp, rho, host_out)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info(dev)
    outs.append(host_out)
    B.sph_diag_sums_noalloc(params, c.n, pos, vel, spin, sp, rho, dev_out)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info(dev)
    assert free_after == free_before
    outs.append(dev_out.cpu().numpy())
    for o in outs:
        assert o[0] == ref["mass"] and o[1] == ref["mass_s"] and o[2] == ref["mass_n"]
        Lscale = np.abs(ref["L_orb"]).max()
        for a in range(3):
            assert _close(o[3 + a], ref["mom"][a], np.abs(ref["mom"]).max() + 1e-300)
            assert _close(o[6 + a], ref["L_orb"][a], Lscale)
            assert _close(o[9 + a], ref["L_spin"][a], np.abs(ref["L_spin"]).max() + 1e-300)
        assert _close(o[12], ref["E_kin"], 0.0)
        assert _close(o[13], ref["E_rot"], 0.0)
        assert _close(o[14], ref["E_int"], abs(ref["E_kin"]))
        assert o[15] == 0.0
        assert o[16] == ref["rho_min"] and o[17] == ref["rho_max"] and o[18] == ref["v_max"]
    assert np.array_equal(outs[0], outs[1])
    # and against the CPU oracle's FP64 diagnostics of the same state
    import oracle
    ref = oracle.diagnostics(oracle.make_params(c.params), st["pos"], st["vel"], st["spin"],
                             c.species, st["rho"])
    o = outs[0]
    assert o[0] == pytest.approx(ref["mass"], rel=TOL)
    assert o[1] == pytest.approx(ref["mass_s"], rel=TOL)
    assert o[2] == pytest.approx(ref["mass_n"], rel=TOL)
    fl = c.species < 2
    m = o[0] / fl.sum()
    vs = m * np.linalg.norm(st["vel"][fl], axis=1).sum()
    ls = m * np.linalg.norm(np.cross(st["pos"][fl], st["vel"][fl]), axis=1).sum()
    ss = np.linalg.norm(st["spin"][fl], axis=1).sum() * m * c.params["inertia_coef"]
    for a in range(3):
        assert abs(o[3 + a] - ref["mom"][a]) <= TOL * vs
        assert abs(o[6 + a] - ref["L_orb"][a]) <= TOL * ls
        assert abs(o[9 + a] - ref["L_spin"][a]) <= TOL * ss + 1e-300
    for k, q in (("E_kin", 12), ("E_rot", 13), ("E_int", 14), ("rho_min", 16),
                 ("rho_max", 17), ("v_max", 18)):
        assert o[q] == pytest.approx(ref[k], rel=TOL, abs=1e-300), k
    sim.close()


def test_noalloc_rejects_oversize_and_host_inputs():
    c = synth.workload("cyl_8960")
    params = B.params_from_dict(c.params)
    out = np.zeros(B.SPH_DIAG_SUMS)
    # host arrays are not accepted as inputs (the kernel reads them directly)
    with pytest.raises(B.SphError) as e:
        B.sph_diag_sums_noalloc(params, c.n, c.pos, c.vel, c.spin, c.species,
                                np.ones(c.n), out)
    assert e.value.status == -1
    import torch
    d = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    # more particles than the fixed scratch array holds
    with pytest.raises(B.SphError) as e:
        B.sph_diag_sums_noalloc(params, 67_108_865, d, d, d, d, d, out)
    assert e.value.status == -1
