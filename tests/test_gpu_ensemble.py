"""The batched ensemble: 64 uneven cylinders (20k..500k fluid particles,
Omega in U(0.05, 0.2), viscous fraction U(0.02, 0.5), R:H in U(0.25, 1))
advanced together by one launch per stage and one CUDA graph per step, in the
mixed form.  Every member must equal its own single-instance run bit for bit,
keep its mass exactly and close its own angular-momentum budget."""
import numpy as np
import pytest

from paper_2405_03980_gb300 import _binding as B
from paper_2405_03980_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


@pytest.mark.parametrize("precision", [B.SPH_MIXED])
def test_ensemble_members_equal_solo_runs(precision):
    from paper_2405_03980_gb300.sim import Simulation
    insts = synth.ensemble(64)
    counts = [c.n for c in insts]
    assert len(insts) == 64 and 5e6 < sum(counts) < 2e7
    ens = Simulation(insts, precision=precision)
    d0 = [ens.diagnostics(k) for k in range(len(insts))]
    ens.step(3)
    st = ens.state_arrays()
    offs = np.concatenate([[0], np.cumsum(counts)])
    for k in range(len(insts)):
        d = ens.diagnostics(k)
        assert d["mass"] == d0[k]["mass"] and d["step"] == 3
        Lz0 = d0[k]["L_orb"][2] + d0[k]["L_spin"][2]
        Lz = d["L_orb"][2] + d["L_spin"][2]
        assert abs(Lz - Lz0 - d["J_wall"][2]) < 1e-5 * abs(Lz0), k
    for k in (0, 17, int(np.argmax(counts)), 63):
        solo = Simulation(insts[k], precision=precision)
        solo.step(3)
        s = solo.state_arrays()
        for f in ("pos", "vel", "spin", "rho", "P", "acc", "dspin"):
            assert np.array_equal(st[f][offs[k]:offs[k + 1]], s[f]), (k, f)
        assert solo.diagnostics(0)["L_orb"] == ens.diagnostics(k)["L_orb"]
        solo.close()
    ens.close()
