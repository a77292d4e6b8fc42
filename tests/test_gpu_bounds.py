"""The bounds-checked build (-DFWI_BOUNDS_CHECK), the stand-in for a memory checker: on
the cases of bounds_cases.py (four meshes: free top, top PML, no PML, thin interior;
forward, stored and checkpointed batched gradients, forward and adjoint rates, a
persistent sweep) no guarded index leaves its range (a failed guard makes the call
return FWI_E_BOUNDS, which fails the child process), and the results equal the normal
build's bit for bit (the guards skip work only when they fail)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(lib, path):
    env = dict(os.environ, FWI_LIBRARY=lib)
    subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py"), path], env=env, check=True, timeout=900)
    return np.load(path)


def test_checked_build_stays_in_bounds_and_matches(tmp_path):
    from paper_1504_08340_gb300 import build

    plain = _run(build.build(), str(tmp_path / "plain.npz"))
    checked = _run(build.build_checked(), str(tmp_path / "checked.npz"))
    assert int(plain["checked"]) == 0 and int(checked["checked"]) == 1
    assert set(plain.files) == set(checked.files)
    for k in plain.files:
        if k != "checked":
            assert np.array_equal(plain[k], checked[k]), k
    # the cases did work: nonzero traces and gradients on every mesh
    for m in range(4):
        assert np.abs(plain[f"m{m}_traces"]).max() > 0 and np.abs(plain[f"m{m}_gl5"]).max() > 0
