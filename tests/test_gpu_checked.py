"""The checked build (-DSPH_CHECKED: device bounds checks on the indices the
kernels take from data, latching SPH_ERR_BOUNDS) runs the whole step without
a failed check and gives the results of the default build, both forms, with
the optional steps on.  The library choice is per process, so the checked
run happens in a child process with SPH_CHECKED=1."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2405_03980_gb300 import _binding as B
from paper_2405_03980_gb300 import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
from paper_2405_03980_gb300 import _binding as B, synth
from paper_2405_03980_gb300.sim import Simulation
lib = B.lib()
assert lib._name.endswith("libsph_gb300_checked.so"), lib._name
out = {}
for prec, extra in ((B.SPH_FP64, 0), (B.SPH_MIXED, B.SPH_PFILTER | B.SPH_COLLISION)):
    c = synth.workload("cyl_8960", seed=6)
    c.params = dict(c.params, col_dist=0.95, flags=B.SPH_FLAGS_DEFAULT | extra)
    s = Simulation(c, precision=prec)
    s.step(5)
    s.check()
    st = s.state_arrays()
    np.savez(sys.argv[1] + f"_{prec}.npz", **st)
    s.close()
print("checked-ok")
'''


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_03980_gb300 import build
    build.build()
    build.build(checked=True)
    yield


def test_checked_build_runs_clean_and_matches(tmp_path):
    from paper_2405_03980_gb300.sim import Simulation
    base = str(tmp_path / "checked")
    env = dict(os.environ, SPH_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD, base], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "checked-ok" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
    for prec, extra, tol in ((B.SPH_FP64, 0, 1e-12),
                             (B.SPH_MIXED, B.SPH_PFILTER | B.SPH_COLLISION, 1e-5)):
        c = synth.workload("cyl_8960", seed=6)
        c.params = dict(c.params, col_dist=0.95, flags=B.SPH_FLAGS_DEFAULT | extra)
        s = Simulation(c, precision=prec)
        s.step(5)
        st = s.state_arrays()
        s.close()
        chk = np.load(base + f"_{prec}.npz")
        for f in st:
            ref = np.abs(st[f]).max()
            err = np.abs(chk[f] - st[f]).max() / (ref if ref > 0 else 1.0)
            assert err <= tol, (prec, f, err)
