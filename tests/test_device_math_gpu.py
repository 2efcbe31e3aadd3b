"""The kernels' own device math against CUDA's functions and float64 (GPU).

atan_poly (the slip-angle arctangent) must stay within 3e-7 relative of the
true arctangent and within 4 float32 ulp of CUDA's atanf, and the paired
arctangent must give its bits on both of its paths; the Pacejka arguments
B steer - B atan(y) must agree with float64; the closed form of
sin(1.5 atan z) used by the Pacejka force (returned without the 1/sqrt(2)
that the host folds into the axle constants) must agree with CUDA's
sinf(1.5f * atanf(z)) and with float64 to 1e-6 relative.
"""

import ctypes
import json
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = str(tmp_path_factory.mktemp("probe") / "libprobe.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-ftz=true", "-shared",
                    "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "paper_2209_12842_gb300", "csrc"),
                    os.path.join(HERE, "cuda", "device_math_probe.cu"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    lib.device_math_probe.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    return lib


def _run(lib, z):
    zt = torch.from_numpy(z.astype(np.float32)).cuda()
    out = torch.empty((z.size, 10), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    assert lib.device_math_probe(zt.data_ptr(), z.size, out.data_ptr()) == 0
    return out.cpu().numpy().astype(np.float64)


def test_atan_poly(probe):
    z = np.concatenate([np.linspace(-4, 4, 400001), np.logspace(-30, 30, 20001), -np.logspace(-30, 30, 20001),
                        [0.0, 1.0, -1.0, np.inf, -np.inf]]).astype(np.float32)
    r = _run(probe, z)
    exact = np.arctan(z.astype(np.float64))
    nz = exact != 0
    rel = np.abs(r[nz, 0] - exact[nz]) / np.abs(exact[nz])
    assert rel.max() < 3e-7, rel.max()
    ulp = np.spacing(np.abs(r[:, 1]).astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(r[:, 0] - r[:, 1]) / np.maximum(ulp, 1e-45)) <= 4
    assert np.isnan(_run(probe, np.array([np.nan]))[0, 0])


def test_pacejka_closed_form(probe):
    z = np.concatenate([np.linspace(-40, 40, 200001), np.logspace(-20, 3, 10001)]).astype(np.float32)
    r = _run(probe, z)
    exact = np.sin(1.5 * np.arctan(z.astype(np.float64)))
    nz = np.abs(exact) > 1e-30
    assert np.max(np.abs(r[nz, 2] - exact[nz]) / np.abs(exact[nz])) < 1e-6
    assert np.max(np.abs(r[nz, 2] - r[nz, 3]) / np.abs(exact[nz])) < 2e-6


def test_atan_pair_paths_are_bitwise_equal(probe):
    # mixed warps (some |z| > 1) take the general path; clamped warps the fast one
    z = np.concatenate([np.linspace(-3, 3, 100001), np.linspace(-1, 1, 100001)]).astype(np.float32)
    r = _run(probe, z).astype(np.float32)
    np.testing.assert_array_equal(r[:, 4], r[:, 0])
    np.testing.assert_array_equal(r[:, 5], r[:, 6])
    np.testing.assert_array_equal(r[:, 7], r[:, 6])


def test_pacejka_arguments(probe):
    # B = 10, B steer = 0.25: the front argument 0.25 - 10 atan(y), the rear -10 atan(0.5)
    z = np.concatenate([np.linspace(-4, 4, 200001), np.logspace(-20, 6, 10001),
                        -np.logspace(-20, 6, 10001)]).astype(np.float32)
    r = _run(probe, z)
    exact = 0.25 - 10.0 * np.arctan(z.astype(np.float64))
    assert np.max(np.abs(r[:, 8] - exact)) < 1e-5
    assert np.max(np.abs(r[:, 9] + 10.0 * np.arctan(0.5))) < 1e-5


@pytest.fixture(scope="module")
def pair_probe(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_12842_gb300 import binding, build

    build.build()
    pkg = os.path.dirname(binding.LIB_PATH)
    out = str(tmp_path_factory.mktemp("pair") / "libpair.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-ftz=true", "-shared",
                    "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2209_12842_gb300", "csrc"),
                    os.path.join(HERE, "cuda", "pair_probe.cu"), "-L", pkg, "-lramppi",
                    "-Xlinker", "-rpath", "-Xlinker", pkg, "-o", out], check=True)
    binding.lib()
    lib = ctypes.CDLL(out)
    lib.pair_probe_run.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return lib, binding


@pytest.mark.parametrize("C", [1.5, 1.3])
def test_pairs_give_the_bits_of_two_scalars(pair_probe, C):
    # one dynamic-model step (6 Heun sub-steps) on float2 pairs against two
    # scalar steps, random states and controls; C = 1.5 takes the closed-form
    # Pacejka shape, other C the library sin/atan
    import ra_scenes as rs

    lib, binding = pair_probe
    mp = list(rs.preset("small_dyn")["model_params"])
    mp[5] = C
    p = rs.preset("small_dyn", model_params=tuple(mp))
    prob = binding.ra_mppi_problem_from(p)
    n = 20000
    words = torch.from_numpy(np.random.default_rng(5).integers(0, 2**32, (n, 8), dtype=np.uint64)
                             .astype(np.uint32).view(np.int32)).cuda()
    out = torch.empty((n, 40), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    assert lib.pair_probe_run(words.data_ptr(), n, ctypes.addressof(prob), out.data_ptr()) == 0
    o = out.cpu().numpy().view(np.uint32)
    f = out.cpu().numpy()
    checks = {"step rollout a": (slice(12, 18), slice(0, 6)), "step rollout b": (slice(18, 24), slice(6, 12)),
              "pacejka": (slice(26, 28), slice(24, 26))}
    bad = {k: float(np.mean(o[:, a] != o[:, b])) for k, (a, b) in checks.items()}
    bad["derivative components"] = f[:, 32:38].mean(axis=0).tolist()
    assert all(v == 0.0 for k, v in bad.items() if k != "derivative components") \
        and not any(bad["derivative components"]), json.dumps(bad)
