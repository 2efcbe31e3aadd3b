"""RA-MPPI controller object over the C ABI.

PyTorch provides the device buffers and the CUDA stream; every update runs
in libramppi.so's kernels through the functions of ``binding`` (which carry
the C names).  Nothing here computes any part of the method.
"""

import numpy as np
import torch

from . import binding as B


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class RaMppi:
    """One RA-MPPI problem instance (one handle) on the current CUDA device.

    problem: a preset dict (see ``ra_scenes.presets``).
    obstacles: (n, 3) array-like of (x, y, r), optional.
    """

    def __init__(self, problem, obstacles=None, keep_risk_costs=False, max_obstacles=None, differentiable=False):
        if not torch.cuda.is_available():
            raise RuntimeError("RaMppi needs a CUDA device (there is no CPU path)")
        self.p = dict(problem)
        n_obs = 0 if obstacles is None else len(obstacles)
        cap = max_obstacles if max_obstacles is not None else max(n_obs, int(self.p.get("n_obs", 0)), 1)
        flags = (B.RA_MPPI_KEEP_RISK_COSTS if keep_risk_costs else 0) | \
            (B.RA_MPPI_DIFFERENTIABLE if differentiable else 0)
        self.keep_risk_costs = keep_risk_costs
        self._prob = B.ra_mppi_problem_from(self.p, flags=flags, max_obstacles=cap)
        self.h = B.ra_mppi_create(self._prob, torch.cuda.current_device())
        self.K, self.M, self.T = int(self.p["K"]), int(self.p["M"]), int(self.p["T"])
        self.nx, self.nu = {0: (4, 2), 1: (6, 2), 2: (1, 1)}[int(self.p["model"])]
        dev = torch.device("cuda", torch.cuda.current_device())
        self.S_tilde = torch.empty(self.K, dtype=torch.float32, device=dev)
        self.cvar = torch.empty(self.K, dtype=torch.float32, device=dev)
        if obstacles is not None:
            self.set_obstacles(obstacles)

    def close(self):
        if getattr(self, "h", None):
            B.ra_mppi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_obstacles(self, xyr):
        arr = np.ascontiguousarray(np.asarray(xyr, dtype=np.float32).reshape(-1, 3))
        B.ra_mppi_set_obstacles(self.h, arr.ctypes.data if arr.size else None, arr.shape[0])

    def step(self, x0, V, V_out=None, stream=None, want_cvar=True):
        """One update on device tensors; returns V+ (a new tensor unless V_out)."""
        assert x0.is_cuda and V.is_cuda and x0.dtype == torch.float32 and V.dtype == torch.float32
        x0 = x0.contiguous()
        V = V.contiguous()
        out = V_out if V_out is not None else torch.empty_like(V)
        B.ra_mppi_step(self.h, x0.data_ptr(), V.data_ptr(), out.data_ptr(), self.S_tilde.data_ptr(),
                       self.cvar.data_ptr() if want_cvar else None, _stream_ptr(stream))
        return out

    def closed_loop_step(self, x, V, collisions=None, shift=True, stream=None):
        """One receding-horizon iteration on a simulated plant; x and V are
        device tensors updated in place (plant state, warm start).
        `collisions`, if given, is an int32 device tensor of 2 counters:
        steps inside an obstacle and steps off the track."""
        assert x.is_cuda and V.is_cuda and x.is_contiguous() and V.is_contiguous()
        assert collisions is None or (collisions.is_cuda and collisions.dtype == torch.int32
                                      and collisions.numel() >= 2)
        B.ra_mppi_closed_loop_step(self.h, x.data_ptr(), V.data_ptr(), self.S_tilde.data_ptr(),
                                   collisions.data_ptr() if collisions is not None else None,
                                   1 if shift else 0, _stream_ptr(stream))

    def step_host(self, x0, V, S_tilde=False, stream=None):
        """One update on host arrays (copies inside); returns V+ (numpy)."""
        x0 = np.ascontiguousarray(np.asarray(x0, dtype=np.float32))
        V = np.ascontiguousarray(np.asarray(V, dtype=np.float32))
        out = np.empty_like(V)
        st = np.empty(self.K, dtype=np.float32) if S_tilde else None
        B.ra_mppi_step_host(self.h, x0.ctypes.data, V.ctypes.data, out.ctypes.data,
                            st.ctypes.data if st is not None else None, _stream_ptr(stream))
        return (out, st) if S_tilde else out

    def workspace(self, stream=None):
        """Copies of U [K,T,nu], S [K], CVaR [K] (and L [K,M] if kept)."""
        dev = self.S_tilde.device
        U = torch.empty((self.K, self.T, self.nu), dtype=torch.float32, device=dev)
        S = torch.empty(self.K, dtype=torch.float32, device=dev)
        cv = torch.empty(self.K, dtype=torch.float32, device=dev)
        L = torch.empty((self.K, self.M), dtype=torch.float32, device=dev) if self.keep_risk_costs else None
        B.ra_mppi_copy_workspace(self.h, U.data_ptr(), S.data_ptr(), cv.data_ptr(),
                                 L.data_ptr() if L is not None else None, _stream_ptr(stream))
        return dict(U=U, S=S, cvar=cv, L=L)

    def importance_weights(self, stream=None):
        """Copy of the last update's importance weights W [K, M] (needs
        keep_risk_costs and importance sampling on)."""
        W = torch.empty((self.K, self.M), dtype=torch.float32, device=self.S_tilde.device)
        B.ra_mppi_copy_weights(self.h, W.data_ptr(), _stream_ptr(stream))
        return W

    @property
    def iteration(self):
        return B.ra_mppi_get_state(self.h)

    @iteration.setter
    def iteration(self, it):
        B.ra_mppi_set_state(self.h, it)

    def status(self):
        return B.ra_mppi_get_status(self.h)

    def set_launch(self, warps_per_block=0, ilp=0, warps_per_sample=0):
        B.ra_mppi_set_launch(self.h, warps_per_block, ilp, warps_per_sample)

    def set_tail_split(self, enable):
        B.ra_mppi_set_tail_split(self.h, enable)

    def launch_plan(self):
        """(grid, first tail block or -1, tail warps per sample, blocks per SM)."""
        return B.ra_mppi_get_launch_plan(self.h)

    def tune(self, x0, V, replays=3):
        """Pick the fastest launch shape on these inputs (results unchanged)."""
        return B.ra_mppi_tune(self.h, x0.contiguous().data_ptr(), V.contiguous().data_ptr(), replays)

    def get_launch(self):
        return B.ra_mppi_get_launch(self.h)

    def set_cost_weights(self, theta):
        """theta = (w_dev, w_speed, gamma, w_obs) for the following updates."""
        B.ra_mppi_set_cost_weights(self.h, [float(v) for v in theta])

    def backward(self, gV_plus, gS_tilde=None, stream=None):
        """VJP of the most recent update: (dV, dtheta) of
        <gV_plus, V+> + <gS_tilde, S~>."""
        gVp = gV_plus.contiguous().float()
        gS = gS_tilde.contiguous().float() if gS_tilde is not None else None
        gV = torch.empty_like(gVp)
        gth = torch.empty(4, dtype=torch.float32, device=gVp.device)
        B.ra_mppi_backward(self.h, gVp.data_ptr(), gS.data_ptr() if gS is not None else None, gV.data_ptr(),
                           gth.data_ptr(), _stream_ptr(stream))
        return gV, gth

    def set_timing_events(self, begin=None, end=None):
        """Record torch.cuda.Event objects around the fused rollout kernel."""
        if begin is None:
            B.ra_mppi_set_timing_events(self.h, None, None)
            return
        for ev in (begin, end):
            if ev.cuda_event == 0:  # torch creates the CUDA event lazily
                ev.record()
        self._timing = (begin, end)
        B.ra_mppi_set_timing_events(self.h, begin.cuda_event, end.cuda_event)


class RaMppiBatch:
    """B RA-MPPI problems updated together (one persistent launch replayed
    from a CUDA graph).  problem: common preset dict; instances: list of dicts
    with K, M, T, max_obstacles, seed, instance_id."""

    def __init__(self, problem, instances):
        if not torch.cuda.is_available():
            raise RuntimeError("RaMppiBatch needs a CUDA device (there is no CPU path)")
        self.p = dict(problem)
        self.inst = [dict(i) for i in instances]
        prob = B.ra_mppi_problem_from(self.p, max_obstacles=1)
        recs = [B.ra_mppi_instance(int(i["K"]), int(i["M"]), int(i["T"]), int(i["max_obstacles"]),
                                   int(i["seed"]) & 0xFFFFFFFFFFFFFFFF, int(i["instance_id"]) & 0xFFFFFFFF, 0)
                for i in self.inst]
        self.b = B.ra_mppi_batch_create(prob, recs, torch.cuda.current_device())
        self.B = len(self.inst)
        self.nx, self.nu = {0: (4, 2), 1: (6, 2), 2: (1, 1)}[int(self.p["model"])]
        self.offsets = B.ra_mppi_batch_layout(self.b, self.B)
        self.ptr_x0, self.ptr_V, self.ptr_V_out, self.ptr_S_tilde = B.ra_mppi_batch_buffers(self.b)
        self.n_V = sum(int(i["T"]) * self.nu for i in self.inst)
        self.n_k = sum(int(i["K"]) for i in self.inst)
        self.n_U = sum(int(i["K"]) * int(i["T"]) * self.nu for i in self.inst)

    def close(self):
        if getattr(self, "b", None):
            B.ra_mppi_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_obstacles(self, i, xyr):
        arr = np.ascontiguousarray(np.asarray(xyr, dtype=np.float32).reshape(-1, 3))
        B.ra_mppi_batch_set_obstacles(self.b, i, arr.ctypes.data if arr.size else None, arr.shape[0])

    def set_inputs(self, x0s, Vs):
        """Per-problem x0 [nx] and V [T_i, nu] into the packed input buffers."""
        x0 = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float32).ravel() for x in x0s]))
        V = np.ascontiguousarray(np.concatenate([np.asarray(v, np.float32).ravel() for v in Vs]))
        B.ra_mppi_batch_write_inputs(self.b, x0.ctypes.data, V.ctypes.data, _stream_ptr(None))
        torch.cuda.synchronize()

    def step(self, stream=None, graph=True):
        if graph:
            B.ra_mppi_step_batched(self.b, _stream_ptr(stream))
        else:
            B.ra_mppi_step_batched_eager(self.b, _stream_ptr(stream))

    def outputs(self):
        """V+ per problem (list of [T_i, nu]) and S~ per problem (list of [K_i])."""
        Vo = np.empty(self.n_V, dtype=np.float32)
        St = np.empty(self.n_k, dtype=np.float32)
        B.ra_mppi_batch_read_outputs(self.b, Vo.ctypes.data, St.ctypes.data, _stream_ptr(None))
        torch.cuda.synchronize()
        Vs, Ss = [], []
        for i, inst in enumerate(self.inst):
            _, vo, ko, _ = self.offsets[i]
            Vs.append(Vo[vo:vo + int(inst["T"]) * self.nu].reshape(int(inst["T"]), self.nu).copy())
            Ss.append(St[ko:ko + int(inst["K"])].copy())
        return Vs, Ss

    def workspace(self):
        U = torch.empty(self.n_U, dtype=torch.float32, device="cuda")
        S = torch.empty(self.n_k, dtype=torch.float32, device="cuda")
        cv = torch.empty(self.n_k, dtype=torch.float32, device="cuda")
        B.ra_mppi_batch_copy_workspace(self.b, U.data_ptr(), S.data_ptr(), cv.data_ptr(), _stream_ptr(None))
        U, S, cv = U.cpu().numpy(), S.cpu().numpy(), cv.cpu().numpy()
        out = []
        for i, inst in enumerate(self.inst):
            _, _, ko, uo = self.offsets[i]
            K, T = int(inst["K"]), int(inst["T"])
            out.append(dict(U=U[uo:uo + K * T * self.nu].reshape(K, T, self.nu), S=S[ko:ko + K],
                            cvar=cv[ko:ko + K]))
        return out

    def set_iteration(self, it):
        B.ra_mppi_batch_set_iteration(self.b, it)

    def status(self):
        return B.ra_mppi_batch_get_status(self.b)

    def tune(self, replays=3):
        return B.ra_mppi_batch_tune(self.b, replays)

    def set_launch(self, warps_per_block, ilp):
        B.ra_mppi_batch_set_launch(self.b, warps_per_block, ilp)

    def get_launch(self):
        return B.ra_mppi_batch_get_launch(self.b)

    def set_timing_events(self, begin=None, end=None):
        """Record torch.cuda.Event objects around the persistent rollout
        kernel of the eager launch (step(graph=False))."""
        if begin is None:
            B.ra_mppi_batch_set_timing_events(self.b, None, None)
            return
        for ev in (begin, end):
            if ev.cuda_event == 0:  # torch creates the CUDA event lazily
                ev.record()
        self._timing = (begin, end)
        B.ra_mppi_batch_set_timing_events(self.b, begin.cuda_event, end.cuda_event)

    def set_diagnostics(self, counter=None):
        """Count the obstacles tested exactly into an int64 device tensor."""
        B.ra_mppi_batch_set_diagnostics(self.b, counter.data_ptr() if counter is not None else None)


class RaMppiUpdate(torch.autograd.Function):
    """(V+, S~) = update(V, theta) of one RA-MPPI step with the hand-written
    adjoint as its backward; theta = (w_dev, w_speed, gamma, w_obs).

    Usage: V_plus, S_tilde = RaMppiUpdate.apply(V, theta, ctl, x0) with ctl a
    RaMppi created with differentiable=True; the backward must run before
    the handle steps again (it differentiates the handle's latest update)."""

    @staticmethod
    def forward(ctx, V, theta, ctl, x0):
        ctl.set_cost_weights(theta.detach().cpu().tolist())
        V_plus = ctl.step(x0.detach(), V.detach().contiguous())
        ctx.ctl = ctl
        ctx.iteration = ctl.iteration
        ctx.v_shape = V.shape
        return V_plus, ctl.S_tilde.clone()

    @staticmethod
    def backward(ctx, gV_plus, gS_tilde):
        if ctx.ctl.iteration != ctx.iteration:
            raise RuntimeError("the RA-MPPI handle stepped again before backward")
        if gV_plus is None:
            gV_plus = torch.zeros(ctx.v_shape, dtype=torch.float32, device=ctx.ctl.S_tilde.device)
        gV, gth = ctx.ctl.backward(gV_plus, gS_tilde)
        return gV, gth, None, None
