"""The allocation-free softmin update against the handle-based update (GPU).

ra_mppi_softmin_update_noalloc serves callers that cannot allocate device
memory where they run the update (a real-time control thread, a host
program with its own memory pool).  This test calls it through the C ABI on
the S~ and U that ra_mppi_step produced, and checks its V+ against that
step's V+ within the update tolerance of the parity tests (abs 1e-5), on two
calls in a row (the second reuses the scratch the first left behind), with
one problem whose grid fits the fixed scratch and one that exceeds the
handle path's block count.  This file is collected last so that a run that
stops at the first failure has already run every other test.
"""

import numpy as np
import pytest

import ra_scenes as rs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_12842_gb300 import build as b

    b.build()


def _check_two_calls(p, obs):
    from paper_2209_12842_gb300 import RaMppi
    from paper_2209_12842_gb300 import binding as B

    stream = torch.cuda.current_stream().cuda_stream
    ctl = RaMppi(p, obs)
    x0 = torch.from_numpy(rs.initial_state(p["model"])).cuda()
    V = torch.from_numpy(rs.random_controls(p["model"], p["T"], p["u_lo"], p["u_hi"], 3)).cuda()
    K, T, nu = ctl.K, ctl.T, ctl.nu
    lam = float(np.float32(p["lam"]))
    for call in range(2):
        V_plus = ctl.step(x0, V)  # existing entry point: S~ and U of this update
        U = ctl.workspace()["U"]
        out = torch.full_like(V_plus, float("nan"))
        rc = B.ra_mppi_softmin_update_noalloc(ctl.S_tilde.data_ptr(), U.data_ptr(), K, T, nu, lam,
                                              out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert rc == B.RA_MPPI_OK, f"call {call}: {B.STATUS_NAMES.get(rc, rc)}"
        np.testing.assert_allclose(out.cpu().numpy(), V_plus.cpu().numpy(), atol=1e-5, rtol=0,
                                   err_msg=f"call {call}")
        V = V_plus  # warm start for the next call
    ctl.close()


def test_noalloc_matches_handle_update_small():
    p = rs.preset("small_kin", K=777)
    _check_two_calls(p, rs.obstacles_ahead(1, 8, 0.15, 0.3))


def test_noalloc_matches_handle_update_beyond_block_cap():
    # 20000 samples: 79 update blocks on the handle path, 64 on the fixed scratch
    p = rs.preset("c3_instance", K=20000, M=16, T=50)
    _check_two_calls(p, rs.make_obstacles(p["seed"], p["n_obs"], *p["obs_r"]))


def test_noalloc_rejects_sizes_beyond_the_limit():
    from paper_2209_12842_gb300 import binding as B

    buf = torch.zeros(600 * 2, device="cuda")
    st = torch.zeros(4, device="cuda")
    assert B.ra_mppi_softmin_update_noalloc(st.data_ptr(), buf.data_ptr(), 4, 257, 2, 1.0,
                                            buf.data_ptr()) == B.RA_MPPI_EINVAL
    assert B.ra_mppi_softmin_update_noalloc(st.data_ptr(), buf.data_ptr(), 0, 10, 2, 1.0,
                                            buf.data_ptr()) == B.RA_MPPI_EINVAL
    assert B.ra_mppi_softmin_update_noalloc(st.data_ptr(), buf.data_ptr(), 4, 10, 2, 0.0,
                                            buf.data_ptr()) == B.RA_MPPI_EINVAL
