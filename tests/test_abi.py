"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/phasorpic.h declares; struct layouts match the binding."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "phasorpic.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(pp_[a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pp_init_cell", "pp_set_circuit_state", "pp_advance_period", "pp_get_turn_phasors",
                     "pp_get_vacuum_impedance", "pp_destroy", "pp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2609_15043_b300 import build_lib
    lib_path = build_lib.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pp_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        getattr(lib, n)


def test_binding_struct_layout():
    from paper_2609_15043_b300 import phasorpic as pp
    assert pp.lib.pp_config_size() == ctypes.sizeof(pp.PPConfig)
    assert pp.lib.pp_record_size() == ctypes.sizeof(pp.PPRecord)
    assert set(pp.EXPORTS) == set(declared_functions())


def test_library_targets_sm_103a():
    from paper_2609_15043_b300 import build_lib
    lib_path = build_lib.build()
    out = subprocess.run(["cuobjdump", "--list-elf", lib_path], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_errors_without_gpu_are_reported_not_raised():
    """No CUDA device here: pp_init_cell returns an error code and a message."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2609_15043_b300 import phasorpic as pp
    from paper_2609_15043_b300 import workloads
    with pytest.raises(pp.PhasorPICError):
        pp.Cell(workloads.small())


def test_config_validation_phase_closure():
    """Eq. phaseclosure: a dt that does not close the period is rejected
    before any device work."""
    from paper_2609_15043_b300 import phasorpic as pp
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small().replace(dt=1.0 / (400.5 * 13.56e6))
    with pytest.raises(pp.PhasorPICError, match="phase closure"):
        pp.Cell(cfg)


@pytest.mark.parametrize("change, message", [
    (dict(nr=600), "nr exceeds"),
    (dict(nz=1200, n_init=10), "nz exceeds"),
    (dict(plain_fp64=2), "plain_fp64"),
    (dict(z_coil=0.128), "coil turn nodes must lie above"),
    (dict(nr=128, nz=192, turn_r=[0.05], winding=[1], wire_radius=0.008), "too many turn nodes"),
])
def test_config_validation_limits(change, message):
    """Sizes and placements the kernels do not support are refused at
    pp_init_cell, before any device work."""
    from paper_2609_15043_b300 import phasorpic as pp
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small().replace(**change)
    with pytest.raises(pp.PhasorPICError, match=message):
        pp.Cell(cfg)
