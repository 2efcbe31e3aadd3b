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

    def __init__(self, problem, obstacles=None, keep_risk_costs=False, max_obstacles=None):
        if not torch.cuda.is_available():
            raise RuntimeError("RaMppi needs a CUDA device (there is no CPU path)")
        self.p = dict(problem)
        n_obs = 0 if obstacles is None else len(obstacles)
        cap = max_obstacles if max_obstacles is not None else max(n_obs, int(self.p.get("n_obs", 0)), 1)
        flags = B.RA_MPPI_KEEP_RISK_COSTS if keep_risk_costs else 0
        self.keep_risk_costs = keep_risk_costs
        self._prob = B.ra_mppi_problem_from(self.p, flags=flags, max_obstacles=cap)
        self.h = B.ra_mppi_create(self._prob)
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

    @property
    def iteration(self):
        return B.ra_mppi_get_iteration(self.h)

    @iteration.setter
    def iteration(self, it):
        B.ra_mppi_set_iteration(self.h, it)

    def status(self):
        return B.ra_mppi_get_status(self.h)

    def set_launch(self, warps_per_block=0, ilp=0):
        B.ra_mppi_set_launch(self.h, warps_per_block, ilp)

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
