"""Uneven batching across solver shapes: one solve call for batches of
different contact models (and horizons), each on its own handle and stream.

Each contact model is its own compiled solver shape, so a batch that mixes
point contacts and foot wrenches is solved as one sub-batch per shape.  The
sub-batches run concurrently on separate streams (their kernels share the
GPU), and ragged horizons inside a sub-batch are handled per instance by
the solver itself.  Host logic only: every step runs in the library's
kernels through the C ABI.
"""
from __future__ import annotations

from typing import Dict, List

from . import pinmpc


class MixedSolver:
    """One handle and one stream per sub-batch shape; `solve` enqueues every
    sub-batch and waits for all of them.  With `classes` each handle runs its
    ADMM rounds per horizon class (mpc_set_horizon_classes)."""

    def __init__(self, batches: List, classes: bool = True, graph: bool = False, **overrides):
        import torch

        self.torch = torch
        self.solvers = [pinmpc.solver_for(b, **overrides) for b in batches]
        for s in self.solvers:
            s.set_graph_mode(graph)  # replay each (B, N, warm start) solve from a captured CUDA graph
        if classes:
            # ragged horizons: each round on CTAs sized for each horizon class
            for s, b in zip(self.solvers, batches):
                s.set_horizon_classes(pinmpc.horizon_classes_for(b.N))
        self.streams = [torch.cuda.Stream() for _ in batches]
        self.shapes = [(b.nx, b.nc, b.contact_dim, b.B, b.N) for b in batches]

    def set_stages(self, inputs: List[Dict]):
        """Device inputs of each sub-batch (pinmpc.device_inputs), in order."""
        for s, st, t, shp in zip(self.solvers, self.streams, inputs, self.shapes):
            s.set_stages(shp[3], shp[4], **t, stream=st)

    def warm_start(self, shift: int = 1):
        """The next solve of every sub-batch starts from its last solution
        moved `shift` stages (mpc_warm_start: a receding-horizon step)."""
        for s, st in zip(self.solvers, self.streams):
            s.warm_start(shift, stream=st)

    def solve(self, wait: bool = True):
        for s, st, shp in zip(self.solvers, self.streams, self.shapes):
            s.solve(shp[3], stream=st)
        if wait:
            for st in self.streams:
                st.synchronize()

    def results(self, device: bool = False) -> List[Dict]:
        """Per sub-batch: xi, u, status, iters, kkt after `solve` (numpy, or
        device tensors with device=True, read on each sub-batch's stream)."""
        torch = self.torch
        out = []
        for s, st, (nx, nc, cd, B, N) in zip(self.solvers, self.streams, self.shapes):
            xi = torch.empty((B, N, nx), device="cuda")
            u = torch.empty((B, N, nc * cd), device="cuda")
            status = torch.empty(B, dtype=torch.int32, device="cuda")
            iters = torch.empty(B, dtype=torch.int32, device="cuda")
            kkt = torch.empty(B, device="cuda")
            s.get_traj(xi, u, status, iters, kkt, None, stream=st)
            if device:
                out.append(dict(xi=xi, u=u, status=status, iters=iters, kkt=kkt))
                continue
            st.synchronize()
            out.append(dict(xi=xi.cpu().numpy(), u=u.cpu().numpy(), status=status.cpu().numpy(),
                            iters=iters.cpu().numpy(), kkt=kkt.cpu().numpy()))
        return out

    def close(self):
        for s in self.solvers:
            s.close()
