"""The allocation-free softmin update (GPU).

ra_mppi_softmin_update_noalloc serves callers that cannot allocate device
memory where they run the update: a controller on a real-time thread, where
cudaMalloc and cudaFree may block and synchronise the device, or a host
program that owns all device memory through its own pool.  It keeps its
block partials in one fixed device array that every call shares.

Checks, all through the C ABI:
  - two calls in a row on the S~ and U of ra_mppi_step (the second reuses
    the scratch the first left behind): V+ equal to that existing entry
    point's V+ and to the FP64 oracle's update on the same S~ and U, abs 1e-5
    (the update tolerance of the parity tests);
  - seeded synthetic S~ and U against the oracle's update: S~ with +inf,
    -inf and NaN entries (weight 0), T nu at the limit of 512 columns, K = 1,
    and more samples than the fixed grid's 64 blocks take at 256 each;
  - every S~ non-finite: V_out comes back bit-unchanged;
  - sizes beyond the limits are refused with EINVAL before any work.
This file is collected last, so a run that stops at the first failure has
already run every other test; it also passes alone in a fresh process.
"""

import numpy as np
import pytest

import oracle
import ra_scenes as rs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ATOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_12842_gb300 import build as b

    b.build()


def _noalloc(S_tilde, U, lam, out):
    from paper_2209_12842_gb300 import binding as B

    K, T, nu = U.shape
    rc = B.ra_mppi_softmin_update_noalloc(S_tilde.data_ptr(), U.data_ptr(), K, T, nu, float(lam),
                                          out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rc


def _check_two_calls(p, obs):
    from paper_2209_12842_gb300 import RaMppi
    from paper_2209_12842_gb300 import binding as B

    ctl = RaMppi(p, obs)
    x0 = torch.from_numpy(rs.initial_state(p["model"])).cuda()
    V = torch.from_numpy(rs.random_controls(p["model"], p["T"], p["u_lo"], p["u_hi"], 3)).cuda()
    lam = float(np.float32(p["lam"]))
    for call in range(2):
        V_plus = ctl.step(x0, V)  # the existing entry point: S~, U and V+ of this update
        U = ctl.workspace()["U"]
        out = torch.full_like(V_plus, float("nan"))
        rc = _noalloc(ctl.S_tilde, U, lam, out)
        assert rc == B.RA_MPPI_OK, f"call {call}: {B.STATUS_NAMES.get(rc, rc)}"
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, V_plus.cpu().numpy(), atol=ATOL, rtol=0, err_msg=f"call {call} vs step")
        want, _ = oracle.update(ctl.S_tilde.cpu().numpy(), U.cpu().numpy(), lam)
        np.testing.assert_allclose(got, want, atol=ATOL, rtol=0, err_msg=f"call {call} vs oracle")
        V = V_plus  # warm start for the next call
    ctl.close()


def test_noalloc_matches_step_and_oracle_small():
    p = rs.preset("small_kin", K=777)
    _check_two_calls(p, rs.obstacles_ahead(1, 8, 0.15, 0.3))


def test_noalloc_matches_step_and_oracle_beyond_block_cap():
    # 20000 samples: 256 update blocks on the handle path, 64 on the fixed scratch
    p = rs.preset("c3_instance", K=20000, M=16, T=50)
    _check_two_calls(p, rs.make_obstacles(p["seed"], p["n_obs"], *p["obs_r"]))


def _synthetic(K, T, nu, seed, spread=3.0):
    rng = np.random.default_rng(seed)
    S = (rng.normal(0.0, spread, K) + 50.0).astype(np.float32)
    U = rng.uniform(-3.0, 3.0, (K, T, nu)).astype(np.float32)
    return S, U


@pytest.mark.parametrize("K,T,nu,lam", [
    (1, 20, 2, 1.0),        # K = 1: V+ = U_0
    (300, 256, 2, 1.0),     # T nu = 512 columns, the limit
    (257, 3, 1, 0.35),      # one control dimension, a ragged last block
    (40000, 7, 2, 2.0),     # 157 blocks' worth of samples on the 64-block grid
])
def test_noalloc_against_oracle_synthetic(K, T, nu, lam):
    from paper_2209_12842_gb300 import binding as B

    S, U = _synthetic(K, T, nu, seed=K + T)
    lam = float(np.float32(lam))
    St, Ut = torch.from_numpy(S).cuda(), torch.from_numpy(U).cuda()
    out = torch.full((T, nu), float("nan"), device="cuda")
    for call in range(2):
        assert _noalloc(St, Ut, lam, out) == B.RA_MPPI_OK
        want, _ = oracle.update(S, U, lam)
        np.testing.assert_allclose(out.cpu().numpy(), want, atol=ATOL, rtol=0, err_msg=f"call {call}")
    if K == 1:
        np.testing.assert_array_equal(out.cpu().numpy(), U[0])


def test_noalloc_non_finite_costs_get_zero_weight():
    from paper_2209_12842_gb300 import binding as B

    K, T, nu = 1000, 12, 2
    S, U = _synthetic(K, T, nu, seed=7)
    S[[0, 5, 999]] = np.inf
    S[[3, 700]] = -np.inf
    S[[11, 512]] = np.nan
    S[17] = S[~np.isnan(S) & np.isfinite(S)].min() - 0.5  # a finite minimum next to them
    St, Ut = torch.from_numpy(S).cuda(), torch.from_numpy(U).cuda()
    out = torch.full((T, nu), float("nan"), device="cuda")
    assert _noalloc(St, Ut, 1.0, out) == B.RA_MPPI_OK
    want, w = oracle.update(S, U, 1.0)
    assert np.all(w[~np.isfinite(S)] == 0.0)
    np.testing.assert_allclose(out.cpu().numpy(), want, atol=ATOL, rtol=0)


def test_noalloc_all_non_finite_leaves_output_untouched():
    from paper_2209_12842_gb300 import binding as B

    K, T, nu = 600, 10, 2
    _, U = _synthetic(K, T, nu, seed=3)
    S = np.full(K, np.inf, np.float32)
    S[::3] = np.nan
    S[1::3] = -np.inf
    pattern = torch.arange(T * nu, dtype=torch.float32, device="cuda").reshape(T, nu) * 0.125 - 1.0
    out = pattern.clone()
    rc = _noalloc(torch.from_numpy(S).cuda(), torch.from_numpy(U).cuda(), 1.0, out)
    assert rc == B.RA_MPPI_OK
    assert torch.equal(out.view(torch.int32), pattern.view(torch.int32))


def test_noalloc_rejects_sizes_beyond_the_limit():
    from paper_2209_12842_gb300 import binding as B

    buf = torch.zeros(600 * 2, device="cuda")
    st = torch.zeros(4, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert B.ra_mppi_softmin_update_noalloc(st.data_ptr(), buf.data_ptr(), 4, 257, 2, 1.0,
                                            buf.data_ptr(), s) == B.RA_MPPI_EINVAL
    assert B.ra_mppi_softmin_update_noalloc(st.data_ptr(), buf.data_ptr(), 0, 10, 2, 1.0,
                                            buf.data_ptr(), s) == B.RA_MPPI_EINVAL
    assert B.ra_mppi_softmin_update_noalloc(st.data_ptr(), buf.data_ptr(), (1 << 24) + 1, 10, 2, 1.0,
                                            buf.data_ptr(), s) == B.RA_MPPI_EINVAL
    assert B.ra_mppi_softmin_update_noalloc(st.data_ptr(), buf.data_ptr(), 4, 10, 2, 0.0,
                                            buf.data_ptr(), s) == B.RA_MPPI_EINVAL
    assert B.ra_mppi_softmin_update_noalloc(st.data_ptr(), buf.data_ptr(), 4, 10, 2, float("inf"),
                                            buf.data_ptr(), s) == B.RA_MPPI_EINVAL
