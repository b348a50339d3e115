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
    (dict(n_harmonics=5), "n_harmonics"),
    (dict(n_harmonics=-1), "n_harmonics"),
    (dict(see_gamma=1.5), "see_gamma"),
    (dict(see_gamma=0.1, see_t_ev=0.0), "see_t_ev"),
    (dict(particle_weights=2), "particle_weights"),
    (dict(sm_every=-1), "sm_every"),
    (dict(sm_every=5), "split-merge needs"),
    (dict(sm_every=5, sm_target=10, sm_min=20, sm_max=30), "split-merge needs"),
    (dict(sm_every=5, sm_target=40, sm_min=20, sm_max=30), "split-merge needs"),
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


def test_trainer_and_tuning_arguments_are_checked_before_the_device():
    """Bad options and NULL handles of the training and tuning entry points
    come back as PP_E_ARG before any device work."""
    import numpy as np
    from paper_2609_15043_b300 import phasorpic as pp
    rows = (256, 256, 256, 32)
    w = [np.zeros((r, 256), np.float32) for r in rows]
    b = [np.zeros(r, np.float32) for r in rows]
    for change in (dict(n_in=0), dict(n_in=257), dict(n_out=0), dict(n_out=33), dict(batch=0), dict(batch=4097),
                   dict(lr=0.0), dict(beta1=1.0), dict(beta2=-0.1), dict(eps=0.0), dict(weight_decay=-1.0)):
        kw = dict(n_in=206, n_out=12, w=w, b=b)
        kw.update(change)
        with pytest.raises(pp.PhasorPICError, match="PP_E_ARG"):
            pp.Trainer(**kw)
    with pytest.raises(ValueError):
        pp.Trainer(206, 12, w[:3] + [np.zeros((16, 256), np.float32)], b)
    lib = pp.lib                                  # PP_E_ARG = -7
    assert lib.pp_trainer_steps(None) == -1
    assert lib.pp_trainer_destroy(None) == -7
    assert lib.pp_trainer_load(None, None, None, 1) == -7
    assert lib.pp_trainer_epoch(None, None, 1, None) == -7
    assert lib.pp_get_tuning(None, None) == -7
    assert lib.pp_set_tuning(None, None) == -7
    assert lib.pp_autotune(None, 1, None, None, None) == -7
    assert lib.pp_batch_autotune(None, 1, None, None, None) == -7
    assert lib.pp_get_control_counters(None, None, None) == -7
    assert lib.pp_wait_selftest(0, None) == -7
    assert lib.pp_get_particle_weights(None, 0, 0, None, None, None) == -7
    assert lib.pp_set_particles_weighted(None, 0, 0, None, None, None, None, None, None, None, None) == -7


def test_vacuum_problem_is_validated_before_the_device():
    """pp_vacuum_impedance refuses sheets off the interior nodes and empty
    problems before any device work."""
    from paper_2609_15043_b300 import phasorpic as pp
    f = 13.56e6
    for sheets in ([(0, 5, 10)], [(40, 5, 10)], [(10, 0, 10)], [(10, 5, 40)], [(10, 20, 10)], []):
        with pytest.raises(pp.PhasorPICError, match="PP_E_CONFIG"):
            pp.vacuum_impedance(40, 40, 0.04, 0.04, f, sheets)
    with pytest.raises(pp.PhasorPICError, match="PP_E_CONFIG"):
        pp.vacuum_impedance(2, 40, 0.04, 0.04, f, [(1, 5, 10)])
