"""The C ABI without a GPU: the library loads, exports every function that
include/pm.h declares, its host helpers agree with the paper's geometry
(Table 3, q_crit of Sec. 2.2.2) and the fixed-point rule, and pm_create_grids
rejects invalid grid systems before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1210_1736_gb300 import pm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = _declared()
    assert len(names) >= 20
    lib = pm.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(pm._SIGS), set(names) ^ set(pm._SIGS)


def test_cell_length_table3(golden_dir):
    rows = [l.split() for l in open(os.path.join(golden_dir, "table3_vertical_resolution.txt"))
            if l.strip() and not l.startswith("#")]
    for row in rows:
        q = float(row[0])
        for N, printed in zip([64, 128, 256, 512], row[1:]):
            lz = pm.cell_length(28000.0, N, q)
            assert lz == O.cell_length(28000.0, N, q)
            if printed == "-":
                assert q < pm.q_crit(3500, 28000, 105000, N)
            else:
                assert int(printed) in (int(np.floor(lz)), int(round(lz)))


def test_fixed_shift_matches_rule():
    for mb in [1.0, 11.35, 0.75, 2.0**40, 3e-7]:
        assert pm.fixed_shift(mb) == O.fixed_shift(mb)
    assert pm.fixed_shift(0.0) == -2**31
    assert pm.fixed_shift(float("nan")) == -2**31


def _galaxy_desc(q=0.25, n=128, r_core=1.5, r_out=6.0, r_sys=32.0, fine=(128, 128, 32), ngal=1):
    w = dict(precision="fp32",
             system=dict(r_sys=r_sys, sys_centre=(0, 0, 0), G=1.0, h000=1.0),
             galaxies=[dict(coarse=(n, n, n, r_sys, 1.0), medium=(n, n, n, r_out, q),
                            fine=(*fine, r_core, 1.0), r_core=r_core, r_out=r_out,
                            centre=(0, 0, 0), recentre=True) for _ in range(ngal)])
    return pm.describe(w, 1.0)


def _create(sysd, gals):
    h = C.c_void_p()
    rc = pm.lib().pm_create_grids(C.byref(sysd), gals, None, C.byref(h))
    if rc == 0:
        pm.lib().pm_destroy(h)
    return rc, h.value


def test_create_rejects_q_below_qcrit():
    rc, h = _create(*_galaxy_desc(q=0.125))
    assert rc == pm.PM_E_QCRIT and h is None
    assert b"q_crit" in pm.lib().pm_last_error()


def test_create_rejects_second_flattened_galaxy():
    sysd, gals = _galaxy_desc(ngal=2)
    rc, _ = _create(sysd, gals)
    assert rc == pm.PM_E_QCRIT


def test_create_rejects_bad_nesting():
    # fine grid covering more than the medium grid
    rc, _ = _create(*_galaxy_desc(r_core=7.0, r_out=6.0))
    assert rc == pm.PM_E_NESTING


def test_create_rejects_non_power_of_two_and_bad_mass():
    sysd, gals = _galaxy_desc()
    gals[0].coarse.nx = 96
    assert _create(sysd, gals)[0] == pm.PM_E_ARG
    sysd, gals = _galaxy_desc()
    sysd.mass_bound = 0.0
    assert _create(sysd, gals)[0] == pm.PM_E_ARG
    sysd, gals = _galaxy_desc()
    sysd.precision = 3
    assert _create(sysd, gals)[0] == pm.PM_E_ARG


def test_null_arguments_are_errors_not_crashes():
    lib = pm.lib()
    assert lib.pm_solve(None) == pm.PM_E_ARG
    assert lib.pm_deposit(None, None) == pm.PM_E_ARG
    assert lib.pm_create_grids(None, None, None, None) == pm.PM_E_ARG


def test_valid_system_without_gpu_fails_loudly():
    """On a machine without a GPU a valid system is refused with PM_E_CUDA:
    there is no CPU fallback."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, h = _create(*_galaxy_desc())
    assert rc == pm.PM_E_CUDA and h is None
