"""Process-wide settings of the library that live on the host (no GPU needed):
the kernel-path thresholds with their documented ranges, the launch mode with
its clamping, and the validation switch.  Each setter returns or keeps the
previous value as its declaration states."""
import ctypes as C

import pytest

import paper_1404_4797_gb300 as S
from paper_1404_4797_gb300 import build as B


@pytest.fixture
def restore():
    B.build()
    S.lib()
    t = S.get_tuning()
    mode = S.set_launch_mode(-1)
    S.set_launch_mode(mode)
    val = S.set_validation(True)
    S.set_validation(val)
    yield
    S.set_tuning(**t)
    S.set_launch_mode(mode)
    S.set_validation(val)


def _set(small, med, mid, seg):
    return S.lib().sclap_set_tuning(C.byref(S.Tuning(small, med, mid, seg)))


def test_default_tuning():
    # a fresh process: the documented defaults
    B.build()
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c",
                          "import paper_1404_4797_gb300 as S; print(S.get_tuning())"],
                         cwd=root, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert eval(out.stdout) == {"small_max": 32, "med_max": 256, "mid_max": 2048,
                                "seg_smem": 6144}


def test_tuning_ranges(restore):
    good = [(4, 4, 512, 64), (8, 256, 1024, 6144), (16, 16, 2048, 100), (32, 256, 4096, 2048),
            (32, 32, 512, 6144)]
    for t in good:
        assert _set(*t) == S.OK
        assert tuple(S.get_tuning().values()) == t
    before = S.get_tuning()
    bad = [(2, 256, 2048, 6144), (12, 256, 2048, 6144), (64, 256, 2048, 6144),
           (32, 16, 2048, 6144), (32, 257, 2048, 6144), (32, 256, 768, 6144),
           (32, 256, 8192, 6144), (32, 256, 2048, 63), (32, 256, 2048, 6145)]
    for t in bad:
        assert _set(*t) == S.EINVAL, t
        assert S.get_tuning() == before  # a rejected setting changes nothing
    assert S.lib().sclap_set_tuning(None) == S.EINVAL
    with pytest.raises(S.SclapError):
        S.set_tuning(32, 256, 3000, 6144)


def test_launch_mode_is_clamped_and_returns_the_previous(restore):
    S.set_launch_mode(0)
    assert S.set_launch_mode(1) == 0
    assert S.set_launch_mode(7) == 1
    assert S.set_launch_mode(-5) == 2
    assert S.set_launch_mode(0) == -1


def test_validation_switch_returns_the_previous(restore):
    S.set_validation(True)
    assert S.set_validation(False) is True
    assert S.set_validation(False) is False
    assert S.set_validation(True) is False
