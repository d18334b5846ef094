"""The COG_DEBUG build (libcog_debug.so): every data-dependent kernel index
is bounds-checked before its access.  A run of every kernel family through
it must end with no failed check (cog_sync would return COG_ERR_DEVICE and
name the check), and its masks must equal libcog.so's: the checks change no
result."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_09339_gb300.build import build
    build(debug=True)


def test_debug_build_runs_clean_and_matches(built, tmp_path):
    out = tmp_path / "dbg.npz"
    env = dict(os.environ, COG_LIB_VARIANT="debug")
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_workload.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    dbg = dict(np.load(out))
    assert int(dbg.pop("debug_build")[0]) == 1
    sys.path.insert(0, HERE)
    import debug_build_workload
    from paper_1705_09339_gb300 import cog
    assert cog.lib.cog_debug_build() == 0
    ref = debug_build_workload.run()
    assert int(ref.pop("debug_build")[0]) == 0
    assert sorted(ref) == sorted(dbg)
    for k in ref:
        assert np.array_equal(ref[k], dbg[k]), k
