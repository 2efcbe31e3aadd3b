"""The C-ABI library builds, loads and exports what include/*.h declares (CPU only).

No compute call is made here: without a GPU the library must still load,
report its struct size, reject invalid problems with EINVAL before touching
CUDA, and fail cleanly (not crash) when no device is present.
"""

import ctypes
import glob
import os
import re

import pytest

import ra_scenes as rs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2209_12842_gb300 import build as b

    b.build()
    import paper_2209_12842_gb300 as p

    p.lib()
    return p


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ra_mppi_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("ra_mppi_create", "ra_mppi_step", "ra_mppi_destroy", "ra_mppi_step_host"):
        assert required in names


# The boundary's calls as the hot-path scope names them: create with a
# device, set obstacles, the single and batched steps, the batch's
# library-owned inputs, the adjoint, the status word, resumable state and
# the error text.  Extra entry points (host-buffer step, closed loop,
# workspace views, tuning, the allocation-free update) sit beside them.
BOUNDARY = ("ra_mppi_create", "ra_mppi_set_obstacles", "ra_mppi_step", "ra_mppi_batch_create",
            "ra_mppi_batch_io", "ra_mppi_step_batched", "ra_mppi_backward", "ra_mppi_get_status",
            "ra_mppi_get_state", "ra_mppi_set_state", "ra_mppi_last_error", "ra_mppi_destroy",
            "ra_mppi_batch_destroy")


def test_header_declares_the_scoped_boundary():
    names = _declared_functions()
    missing = [n for n in BOUNDARY if n not in names]
    assert not missing, missing
    text = open(os.path.join(ROOT, "include", "ra_mppi.h")).read()
    # create and batch_create take the device they bind the handle to
    assert re.search(r"int ra_mppi_create\(const ra_mppi_problem\* p, int32_t device, ra_mppi_t\*\* out\)", text)
    assert re.search(r"int ra_mppi_batch_create\([^)]*int32_t B, int32_t device,", text)


def test_library_exports_every_declared_symbol(pkg):
    lib = ctypes.CDLL(pkg.binding.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_problem_struct_layout(pkg):
    assert pkg.lib().ra_mppi_problem_size() == ctypes.sizeof(pkg.binding.ra_mppi_problem)


@pytest.mark.parametrize("field,value", [
    ("K", 0), ("M", 513), ("T", 0), ("lam", 0.0), ("alpha", 1.0), ("alpha", 0.0),
    ("B", -1.0), ("eta", 1.0), ("substeps", 0), ("model", 7), ("cvar_mode", 6),
])
def test_create_rejects_invalid_problems(pkg, field, value):
    p = rs.preset("c1_plain", **{field: value})
    prob = pkg.binding.ra_mppi_problem_from(p)
    with pytest.raises(pkg.binding.RaMppiError) as ei:
        pkg.binding.ra_mppi_create(prob)
    assert ei.value.code == pkg.binding.RA_MPPI_EINVAL


@pytest.mark.parametrize("kappa", [-1.0, float("inf"), float("nan")])
def test_create_rejects_invalid_mean_variance_weight(pkg, kappa):
    p = rs.preset("c1_plain", cvar_mode=rs.RISK_MEANVAR, risk_param=kappa)
    with pytest.raises(pkg.binding.RaMppiError) as ei:
        pkg.binding.ra_mppi_create(pkg.binding.ra_mppi_problem_from(p))
    assert ei.value.code == pkg.binding.RA_MPPI_EINVAL


@pytest.mark.parametrize("ov", [dict(is_scale=0.5, is_frac=0.5), dict(is_scale=17.0, is_frac=0.5),
                                dict(is_scale=float("nan"), is_frac=0.5), dict(is_scale=2.0, is_frac=1.0),
                                dict(is_scale=2.0, is_frac=-0.1),
                                dict(is_scale=2.0, is_frac=0.5, noise_type=rs.NOISE_UNIFORM),
                                dict(is_scale=2.0, is_frac=0.5, noise_type=rs.NOISE_IMPULSE)])
def test_create_rejects_invalid_importance_sampling(pkg, ov):
    p = rs.preset("c1_plain", **ov)
    with pytest.raises(pkg.binding.RaMppiError) as ei:
        pkg.binding.ra_mppi_create(pkg.binding.ra_mppi_problem_from(p))
    assert ei.value.code == pkg.binding.RA_MPPI_EINVAL


def test_batched_path_validates_importance_sampling(pkg):
    p = rs.preset("c1_plain", is_scale=1.5, is_frac=0.5, noise_type=rs.NOISE_UNIFORM)
    inst = [pkg.binding.ra_mppi_instance(K=64, M=32, T=10, max_obstacles=4, seed=1, instance_id=0, reserved=0)]
    with pytest.raises(pkg.binding.RaMppiError) as ei:
        pkg.binding.ra_mppi_batch_create(pkg.binding.ra_mppi_problem_from(p), inst)
    assert ei.value.code == pkg.binding.RA_MPPI_EINVAL


def test_null_arguments(pkg):
    L = pkg.lib()
    assert L.ra_mppi_create(None, -1, None) == pkg.binding.RA_MPPI_EINVAL
    assert L.ra_mppi_step(None, None, None, None, None, None, None) == pkg.binding.RA_MPPI_EINVAL
    L.ra_mppi_destroy(None)
    assert L.ra_mppi_last_error(None) == b"null handle"


def test_create_without_gpu_fails_cleanly(pkg):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    prob = pkg.binding.ra_mppi_problem_from(rs.preset("c1_plain"))
    with pytest.raises(pkg.binding.RaMppiError) as ei:
        pkg.binding.ra_mppi_create(prob)
    assert ei.value.code in (pkg.binding.RA_MPPI_ECUDA, pkg.binding.RA_MPPI_ENOMEM)


def test_injected_allocation_failure(pkg, monkeypatch):
    monkeypatch.setenv("RAMPPI_FAULT", "alloc")
    prob = pkg.binding.ra_mppi_problem_from(rs.preset("c1_plain"))
    with pytest.raises(pkg.binding.RaMppiError) as ei:
        pkg.binding.ra_mppi_create(prob)
    assert ei.value.code == pkg.binding.RA_MPPI_ENOMEM


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_2209_12842_gb300.binding as B

    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        B.lib()
