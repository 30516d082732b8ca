"""The C-ABI library loads and exports every symbol include/smc2.h declares, and its
host-side validation works without a GPU (no device calls are made here)."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "smc2.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2407_17296_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("no nvcc to build the library")
        build.build_library()
    return binding.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b([a-z_0-9]+)\s*\([^;{]*\)\s*;", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("smc2_create", "pf_loglik_grad", "smc2_step", "smc2_submit", "smc2_poll",
                     "smc2_destroy", "smc2_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2407_17296_gb300 import binding
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in binding.EXPORTS, name


def test_config_layout_matches(lib):
    from paper_2407_17296_gb300 import binding
    c = binding.Config()
    lib.smc2_config_init(ctypes.byref(c))
    assert c.struct_size == ctypes.sizeof(binding.Config)
    assert c.ess_frac == pytest.approx(0.5) and c.pf_resample == binding.SYSTEMATIC


def _cfg(**kw):
    from paper_2407_17296_gb300 import binding, workloads
    w = workloads.lg4(T=50, N=16, M=64)
    return binding.config_for(w, **kw)


def test_footprint_scales_with_sizes(lib):
    from paper_2407_17296_gb300 import binding
    b1 = binding.footprint(_cfg(ckpt_every=1))
    b4 = binding.footprint(_cfg(ckpt_every=4))
    assert b1 > b4 > 0
    # trajectory of (x, log w) for every step dominates at ckpt_every = 1
    N, M, T, dx = 16, 64, 50, 4
    assert b1 >= N * (T + 1) * M * (4 * dx + 4) + N * T * M * 2


@pytest.mark.parametrize("field,value,code", [
    ("D", 7, -1), ("M", 5000, -1), ("N", 0, -1), ("T", 0, -1), ("ess_frac", 1.5, -1),
    ("pf_resample", 3, -1), ("proposal", 9, -1), ("gamma", 0.0, -1), ("particles_per_thread", 3, -1),
    ("d_x", 3, -1), ("struct_size", 12, -1), ("model_family", 7, -1)])
def test_invalid_configs_are_rejected(lib, field, value, code):
    from paper_2407_17296_gb300 import binding
    c = _cfg()
    setattr(c, field, value)
    b = ctypes.c_size_t(0)
    assert lib.smc2_footprint(ctypes.byref(c), ctypes.byref(b)) == code
    assert len(binding.last_error()) > 0


def test_null_arguments_are_rejected(lib):
    assert lib.smc2_destroy(None) == -1
    assert lib.smc2_step(None, None) == -1
    assert lib.pf_loglik_grad(None, None, 1, 1, None, None) == -1
    assert lib.smc2_poll(None, 1, None) == -1
    h = ctypes.c_void_p()
    assert lib.smc2_create(None, ctypes.byref(h)) == -1


def test_server_rejects_bad_arguments_without_device(lib):
    s = ctypes.c_void_p()
    assert lib.smc2_server_create(0, 1, ctypes.byref(s)) == -1
    assert lib.smc2_server_create(1 << 30, 0, ctypes.byref(s)) == -1


@pytest.mark.parametrize("M,ok", [(1024, True), (2048, True), (3000, False), (4096, False)])
def test_shared_memory_limit_of_the_16_dim_model(lib, M, ok):
    """A 16-dimensional filter block holds M x 16 staged states: M = 2048 fits (the adjoint
    then reads slices from memory instead of a ring), M = 3000 does not and is refused."""
    from paper_2407_17296_gb300 import binding, workloads
    w = workloads.lg16(T=20, N=4, M=M)
    c = binding.config_for(w)
    b = ctypes.c_size_t(0)
    rc = lib.smc2_footprint(ctypes.byref(c), ctypes.byref(b))
    if ok:
        assert rc == 0 and b.value > 0
    else:
        assert rc == -1 and "too large" in binding.last_error()


def test_set_launch_validates_without_device(lib):
    from paper_2407_17296_gb300 import binding, workloads
    c = binding.config_for(workloads.lg4(T=20, N=4, M=256))
    with pytest.raises(binding.Smc2Error):
        binding.set_launch(c, [3, 64, 2, 64, 1])    # no 3-particle variant
    with pytest.raises(binding.Smc2Error):
        binding.set_launch(c, [2, 64, 2, 64, 0])    # checkpoint interval outside [1, T]
    binding.set_launch(c, [2, 64, 4, 128, 5])


@pytest.mark.parametrize("steps,code", [(0, -1), (65, -1), (1, 0), (3, 0), (64, 0)])
def test_hmc_steps_are_validated(lib, steps, code):
    """The HMC proposal takes 1..64 leapfrog steps; other proposals ignore the field."""
    from paper_2407_17296_gb300 import binding
    c = _cfg(proposal=binding.HMC, hmc_steps=steps)
    b = ctypes.c_size_t(0)
    assert lib.smc2_footprint(ctypes.byref(c), ctypes.byref(b)) == code
    c = _cfg(proposal=binding.LANGEVIN, hmc_steps=steps)
    assert lib.smc2_footprint(ctypes.byref(c), ctypes.byref(b)) == 0


def test_new_entry_points_validate_without_device_work(lib):
    """Argument checks of the self-test, stream and static-status calls (no device call)."""
    from paper_2407_17296_gb300 import binding
    assert lib.smc2_selftest_crn(None, None, -1, None, None, None, None) == -1
    assert lib.smc2_selftest_crn(None, None, 4, None, None, None, None) == -1
    assert lib.smc2_get_stream(None, None) == -1
    assert lib.pf_static_get_status(None, None, 0) == -1
    assert "NULL" in binding.last_error() or "status" in binding.last_error()


def test_stats_struct_carries_near_tie_counts():
    from paper_2407_17296_gb300 import binding
    names = [f[0] for f in binding.Stats._fields_]
    assert names[-3:] == ["pf_near_ties", "pf_resample_steps", "outer_near_ties"]
    src = open(HEADER).read()
    for n in names:
        assert re.search(r"\b" + n + r"\s*;", src), n


def test_batch_entry_points_validate_without_device_work(lib):
    import ctypes as C
    out = C.c_void_p()
    assert lib.smc2_batch_create(0, C.byref(out)) == -1
    assert lib.smc2_batch_create(5000, C.byref(out)) == -1
    assert lib.smc2_batch_destroy(None) == -1
    assert lib.smc2_batch_step(None, None, 1, None) == -1
    assert lib.smc2_server_set_fused(None, 1) == -1


@pytest.mark.parametrize("depth,weight,code", [(0, 0, -1), (7, 0, -1), (1, 0, 0), (3, 1, 0), (6, 0, 0),
                                               (3, 2, -1), (3, -1, -1)])
def test_nuts_fields_are_validated(lib, depth, weight, code):
    """The NUTS proposal takes 1..6 doublings and one of its two L-kernels; the footprint grows
    by the per-sample trajectory state ((16 + 2J) D + 9 doubles and the trace)."""
    from paper_2407_17296_gb300 import binding
    c = _cfg(proposal=binding.NUTS, nuts_max_depth=depth, nuts_weight=weight)
    b = ctypes.c_size_t(0)
    assert lib.smc2_footprint(ctypes.byref(c), ctypes.byref(b)) == code
    if code == 0:
        b0 = ctypes.c_size_t(0)
        assert lib.smc2_footprint(ctypes.byref(_cfg(proposal=binding.LANGEVIN)), ctypes.byref(b0)) == 0
        assert b.value > b0.value


def test_nuts_trace_and_point_trace_validate_arguments(lib):
    """The verification calls refuse a NULL handle without any device work."""
    assert lib.smc2_get_nuts_trace(None, None, None, None, None) == -1
    assert lib.smc2_set_point_trace(None, 1) == -1
    assert lib.smc2_get_point_trace(None, 0, None, None) == -1
