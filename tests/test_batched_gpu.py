"""Batched path (ra_mppi_step_batched) against the single-problem path and the oracle.

Every problem of a batch runs the same per-sample device functions as a
single-problem handle, with the same inputs, counters and update-block
partition, so U, S, CVaR, S~ and V+ must be bitwise equal to B separate
ra_mppi_step calls, whatever the launch shape and whether the graph or the
eager launch runs.  A few problems are also checked stage-wise against the
oracle.
"""

import numpy as np
import pytest

import oracle
import ra_scenes as rs
from parity_util import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_12842_gb300 import build as b

    b.build()


def _uneven(n, seed, model):
    rng = np.random.default_rng(seed)
    sizes = [(1, 1, 1), (5, 16, 3), (77, 33, 13), (300, 256, 7), (64, 64, 30), (129, 100, 11)]
    out = []
    for i in range(n):
        K, M, T = sizes[i] if i < len(sizes) else (int(rng.integers(1, 400)), int(rng.choice([16, 32, 64, 128, 256])),
                                                   int(rng.integers(1, 40)))
        n_obs = int(rng.integers(0, 25))
        out.append(dict(K=K, M=M, T=T, max_obstacles=max(n_obs, 1), n_obs=n_obs, seed=rs.BASE_SEED + i,
                        instance_id=i))
    return out


def _setup(name, insts, **ov):
    from paper_2209_12842_gb300.controller import RaMppiBatch

    p = rs.preset(name, **ov)
    model = p["model"]
    batch = RaMppiBatch(p, insts)
    obs, x0s, Vs = [], [], []
    for i, d in enumerate(insts):
        o = rs.obstacles_ahead(100 + i, d["n_obs"], 0.15, 0.3, x_from=0.1 if model == 1 else 0.3,
                               x_to=1.2 if model == 1 else 2.5) if d["n_obs"] else np.zeros((0, 3), np.float32)
        obs.append(o)
        batch.set_obstacles(i, o)
        x0s.append(rs.initial_state(model))
        Vs.append(rs.random_controls(model, d["T"], p["u_lo"], p["u_hi"], 200 + i))
    batch.set_inputs(x0s, Vs)
    return p, batch, obs, x0s, Vs


def _single(p, d, obs, x0, V, iteration):
    from paper_2209_12842_gb300 import RaMppi

    q = dict(p, K=d["K"], M=d["M"], T=d["T"], seed=d["seed"], instance_id=d["instance_id"], n_obs=d["n_obs"])
    ctl = RaMppi(q, obs, max_obstacles=d["max_obstacles"])
    ctl.iteration = iteration
    Vp = ctl.step(torch.from_numpy(x0).cuda(), torch.from_numpy(V).cuda())
    ws = ctl.workspace()
    torch.cuda.synchronize()
    g = dict(V_plus=Vp.cpu().numpy(), S_tilde=ctl.S_tilde.cpu().numpy(), cvar=ws["cvar"].cpu().numpy(),
             U=ws["U"].cpu().numpy(), S=ws["S"].cpu().numpy())
    ctl.close()
    return q, g


def _batch_results(batch):
    Vs, Ss = batch.outputs()
    ws = batch.workspace()
    return [dict(V_plus=Vs[i], S_tilde=Ss[i], **ws[i]) for i in range(batch.B)]


@pytest.mark.parametrize("name,ov", [("small_kin", {}), ("small_dyn", {}),
                                     ("small_kin", dict(is_scale=1.3, is_frac=0.5)),
                                     ("small_dyn", dict(is_scale=1.2, is_frac=0.25))])
def test_batched_equals_single_problems(name, ov):
    # (with importance sampling: per-problem proposal counts and weights)
    insts = _uneven(10, 5, rs.preset(name)["model"])
    p, batch, obs, x0s, Vs = _setup(name, insts, **ov)
    batch.set_iteration(4)
    batch.step()
    res = _batch_results(batch)
    assert batch.status() == 0
    for i, d in enumerate(insts):
        q, g = _single(p, d, obs[i], x0s[i], Vs[i], 4)
        for key in ("U", "S", "cvar", "S_tilde", "V_plus"):
            np.testing.assert_array_equal(res[i][key], g[key], err_msg=f"problem {i} {key}")
    # stage-wise oracle parity on three problems
    for i in (2, 3, 5):
        d = insts[i]
        q = dict(p, K=d["K"], M=d["M"], T=d["T"], seed=d["seed"], instance_id=d["instance_id"])
        ref = oracle.samples(q, x0s[i], Vs[i], obs[i], iteration=4, n_threads=8)
        compare(q, dict(res[i], L=None), ref)
    batch.close()


def test_graph_eager_shapes_and_tuner_agree():
    insts = _uneven(14, 9, 0)
    p, batch, obs, x0s, Vs = _setup("small_kin", insts)
    batch.set_iteration(0)
    batch.step(graph=True)
    base = _batch_results(batch)
    variants = [("eager", None), ("shape", (2, 1)), ("shape", (8, 2)), ("tune", None)]
    for kind, arg in variants:
        if kind == "shape":
            batch.set_launch(*arg)
        elif kind == "tune":
            ms = batch.tune(2)
            assert ms > 0
        batch.set_iteration(0)
        batch.step(graph=(kind != "eager"))
        res = _batch_results(batch)
        for i in range(batch.B):
            for key in ("U", "S", "cvar", "S_tilde", "V_plus"):
                np.testing.assert_array_equal(res[i][key], base[i][key], err_msg=f"{kind} {arg} problem {i} {key}")
    batch.close()


def test_replays_advance_the_counters():
    insts = _uneven(4, 3, 0)
    p, batch, obs, x0s, Vs = _setup("small_kin", insts)
    batch.set_iteration(0)
    batch.step()
    first = _batch_results(batch)
    batch.step()
    second = _batch_results(batch)
    assert not np.array_equal(first[3]["U"], second[3]["U"])
    q, g = _single(p, insts[3], obs[3], x0s[3], Vs[3], 1)
    np.testing.assert_array_equal(second[3]["U"], g["U"])
    np.testing.assert_array_equal(second[3]["V_plus"], g["V_plus"])
    batch.close()


def test_uneven_batch_workload_sampled():
    """The batched workload's size mix (B = 256, K 512..8192, M 16..256,
    T 20..60, 5..60 obstacles): four problems bitwise against separate
    handles, and eight against the oracle stage by stage, among them the
    largest-K problem with M = 256 (every sample of the smallest one, which
    also gives the end-to-end V+ against the oracle's own update)."""
    import os

    from paper_2209_12842_gb300.controller import RaMppiBatch

    insts = rs.batched_instances(256)
    for d in insts:
        d["max_obstacles"] = d["n_obs"]
    p = rs.preset("c3_instance")
    batch = RaMppiBatch(p, insts)
    obs, x0s, Vs = [], [], []
    for i, d in enumerate(insts):
        o = rs.make_obstacles(d["seed"], d["n_obs"], 0.3, 0.3)
        obs.append(o)
        batch.set_obstacles(i, o)
        x0s.append(rs.initial_state(0))
        Vs.append(rs.random_controls(0, d["T"], p["u_lo"], p["u_hi"], d["seed"]))
    batch.set_inputs(x0s, Vs)
    batch.set_iteration(0)
    batch.step()
    res = _batch_results(batch)
    assert batch.status() == 0
    for i in (0, 17, 128, 255):
        q, g = _single(p, insts[i], obs[i], x0s[i], Vs[i], 0)
        for key in ("U", "S", "cvar", "S_tilde", "V_plus"):
            np.testing.assert_array_equal(res[i][key], g[key], err_msg=f"problem {i} {key}")
    big = max((i for i, d in enumerate(insts) if d["M"] == 256), key=lambda i: insts[i]["K"])
    assert insts[big]["K"] >= 6000
    small = min(range(len(insts)), key=lambda i: insts[i]["K"] * insts[i]["M"] * insts[i]["T"])
    rng = np.random.default_rng(3)
    others = [int(i) for i in rng.choice([i for i in range(len(insts)) if i not in (big, small)], 6,
                                         replace=False)]
    threads = os.cpu_count() or 8
    for i in [big, small] + others:
        d = insts[i]
        q = dict(p, K=d["K"], M=d["M"], T=d["T"], seed=d["seed"], instance_id=d["instance_id"])
        if i == small:
            ks = None
        else:
            ks = np.unique(np.concatenate([[0, d["K"] // 2, d["K"] - 1], rng.integers(0, d["K"], 5)])).astype(np.int32)
        ref = oracle.samples(q, x0s[i], Vs[i], obs[i], ks=ks, n_threads=threads)
        compare(q, dict(res[i], L=None), ref, check_update=True)
        print(f"batched problem {i}: K={d['K']} M={d['M']} T={d['T']} obstacles {d['n_obs']}, "
              f"{len(ref['ks'])} samples against the oracle")
    batch.close()


def test_batch_io_gives_the_buffers_and_layout():
    """ra_mppi_batch_io returns the library-owned packed input buffers and
    the per-problem offsets that ra_mppi_batch_buffers and
    ra_mppi_batch_layout give piecewise; writing x0 and V through its
    pointers feeds the next step."""
    from paper_2209_12842_gb300 import binding as B

    insts = _uneven(3, 11, 0)
    p, batch, obs, x0s, Vs = _setup("small_kin", insts)
    x0_ptr, V_ptr, offs = B.ra_mppi_batch_io(batch.b, batch.B)
    assert x0_ptr == batch.ptr_x0 and V_ptr == batch.ptr_V
    assert offs == [tuple(o) for o in batch.offsets]
    batch.set_iteration(0)
    batch.step()
    ref = _batch_results(batch)
    # the same inputs written again through the io pointers give the same step
    nx, nu = batch.nx, batch.nu
    x_all = torch.from_numpy(np.concatenate([np.asarray(x, np.float32).ravel() for x in x0s])).cuda()
    V_all = torch.from_numpy(np.concatenate([np.asarray(V, np.float32).ravel() for V in Vs])).cuda()
    for i, (xo, vo, _, _) in enumerate(offs):
        assert xo == i * nx and vo == sum(int(d["T"]) for d in insts[:i]) * nu

    class _DevView:  # a float32 device vector at a raw pointer (CUDA array interface)
        def __init__(self, ptr, n):
            self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3}

    torch.cuda.synchronize()
    torch.as_tensor(_DevView(x0_ptr, x_all.numel()), device="cuda").copy_(x_all)
    torch.as_tensor(_DevView(V_ptr, V_all.numel()), device="cuda").copy_(V_all)
    torch.cuda.synchronize()
    batch.set_iteration(0)
    batch.step()
    got = _batch_results(batch)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a["V_plus"], b["V_plus"])
    batch.close()
