"""Receding-horizon loop on the GPU (ra_mppi_closed_loop_step) against the oracle.

A closed loop diverges between FP32 and FP64 after a while (discrete costs,
feedback), so every iteration n is replayed stage-wise from the GPU's own
state x_n, warm start V_n and iteration n:
  - per-sample S~ of the update (banded, as in the parity tests),
  - V+ from the GPU's S~ and U through the oracle's update (abs 1e-5), which
    must equal the GPU's next warm start (shifted or not),
  - the plant step x_{n+1} = F(x_n, v0+) + w_n with the plant's noise stream,
  - the collision count over the run.
"""

import numpy as np
import pytest

import oracle
import ra_scenes as rs
from parity_util import check_banded

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_12842_gb300 import build as b

    b.build()


def _run(name, n_updates, shift, obs, **ov):
    from paper_2209_12842_gb300 import RaMppi

    p = rs.preset(name, **ov)
    ctl = RaMppi(p, obs)
    x = torch.from_numpy(rs.initial_state(p["model"])).cuda()
    V = torch.from_numpy(rs.zero_controls(p["model"], p["T"])).cuda()
    hits = torch.zeros(2, dtype=torch.int32, device="cuda")  # obstacle hits, track exits
    rec = []
    for n in range(n_updates):
        x_n, V_n = x.cpu().numpy().copy(), V.cpu().numpy().copy()
        ctl.closed_loop_step(x, V, hits, shift=shift)
        ws = ctl.workspace()
        torch.cuda.synchronize()
        rec.append(dict(x=x_n, V=V_n, x_next=x.cpu().numpy().copy(), V_next=V.cpu().numpy().copy(),
                        S_tilde=ctl.S_tilde.cpu().numpy(), U=ws["U"].cpu().numpy()))
    status = ctl.status()
    ctl.close()
    return p, rec, hits.cpu().numpy(), status


@pytest.mark.parametrize("name,shift", [("small_kin", True), ("small_kin", False), ("small_dyn", True)])
def test_closed_loop_replayed_stagewise(name, shift):
    model = rs.preset(name)["model"]
    obs = rs.obstacles_ahead(3, 10, 0.15, 0.3, x_from=0.1 if model == 1 else 0.2,
                             x_to=1.0 if model == 1 else 2.0)
    p, rec, hits, status = _run(name, 10, shift, obs, K=96, M=32)
    assert status == 0
    lam = float(np.float32(p["lam"]))
    want_hits = np.zeros(2, dtype=np.int64)
    for n, r in enumerate(rec):
        ref = oracle.samples(p, r["x"], r["V"], obs, iteration=n, n_threads=8)
        check_banded("S_tilde", r["S_tilde"], ref["S_tilde"], ref["St_lo"], ref["St_hi"])
        Vp, _ = oracle.update(r["S_tilde"].astype(np.float64), r["U"].astype(np.float64), lam)
        want_V = np.concatenate([Vp[1:], Vp[-1:]], 0) if shift else Vp
        np.testing.assert_allclose(r["V_next"], want_V, atol=1e-5, rtol=0)
        x_ref, hit = oracle.plant_step(p, r["x"].astype(np.float64), Vp[0], n, obs)
        np.testing.assert_allclose(r["x_next"], x_ref, rtol=1e-4, atol=1e-5)
        want_hits += hit
    np.testing.assert_array_equal(hits, want_hits)
    # the plant moved (with obstacles just ahead the controller may back off)
    assert np.linalg.norm(rec[-1]["x_next"][:2] - rec[0]["x"][:2]) > 0.01


def test_closed_loop_is_deterministic_and_resumable():
    from paper_2209_12842_gb300 import RaMppi

    obs = rs.make_obstacles(1, 10, 0.3, 0.3)
    p, rec_a, hits_a, _ = _run("small_kin", 6, True, obs)
    _, rec_b, hits_b, _ = _run("small_kin", 6, True, obs)
    for a, b in zip(rec_a, rec_b):
        np.testing.assert_array_equal(a["x_next"], b["x_next"])
        np.testing.assert_array_equal(a["V_next"], b["V_next"])
    np.testing.assert_array_equal(hits_a, hits_b)
    # resume at iteration 3 from the recorded state and warm start
    ctl = RaMppi(p, obs)
    ctl.iteration = 3
    x = torch.from_numpy(rec_a[3]["x"]).cuda()
    V = torch.from_numpy(rec_a[3]["V"]).cuda()
    ctl.closed_loop_step(x, V)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.cpu().numpy(), rec_a[3]["x_next"])
    np.testing.assert_array_equal(V.cpu().numpy(), rec_a[3]["V_next"])
    ctl.close()


@pytest.mark.parametrize("name", ["small_kin", "small_dyn"])
def test_closed_loop_replays_from_a_cuda_graph(name):
    """The receding-horizon step allocates nothing and never synchronises, so
    a CUDA graph captured around it replays it: the device-side update
    counter advances on each replay and the states, warm starts and collision
    counts equal those of the same number of eager calls, bit for bit."""
    from paper_2209_12842_gb300 import RaMppi

    p = rs.preset(name)
    obs = rs.obstacles_ahead(2, int(p["n_obs"]), *p["obs_r"], x_from=0.1, x_to=1.5)
    runs = {}
    for mode in ("eager", "graph"):
        ctl = RaMppi(p, obs)
        x = torch.from_numpy(rs.initial_state(p["model"])).cuda()
        V = torch.from_numpy(rs.zero_controls(p["model"], p["T"])).cuda()
        hits = torch.zeros(2, dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            ctl.closed_loop_step(x, V, hits)  # first call outside the capture
        torch.cuda.synchronize()
        if mode == "graph":
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                ctl.closed_loop_step(x, V, hits)
            step = g.replay
        else:
            def step():
                ctl.closed_loop_step(x, V, hits)
        with torch.cuda.stream(s):
            for _ in range(25):
                step()
        torch.cuda.synchronize()
        runs[mode] = (x.cpu().numpy(), V.cpu().numpy(), hits.cpu().numpy(), ctl.iteration)
        ctl.close()
    e, g = runs["eager"], runs["graph"]
    for a, b in zip(e[:3], g[:3]):
        np.testing.assert_array_equal(a, b)
    assert e[3] == g[3] == 26
