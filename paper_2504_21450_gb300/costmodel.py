"""The learned cost model: traces of per-tile features and block counts from the
solver, training of the MLP with the library's own kernels, and the pool capacity of a
captured step sequence (argument marshalling only; every step runs in libvlgt).

The paper weighs spatial cells by their velocity-space complexity for load balancing
(Section 2) and notes that ghost cells change that cost (Section 5).  Here the model
predicts, per tile of cells, the largest number of blocks the tile holds in the union
layouts of the next `horizon` steps, from features of the present state; the sum over
tiles sizes the pools of a captured sequence of that many steps.  It never changes f.
"""
from __future__ import annotations

import numpy as np

from . import inputs, vlasov


class Trace:
    """Features and union block counts of consecutive states of one run."""

    def __init__(self, edge: int):
        self.edge = edge
        self.features = []
        self.unions = []

    def record(self, grid: vlasov.Grid) -> None:
        f, u = grid.tile_features(self.edge)
        self.features.append(f)
        self.unions.append(u)

    def dataset(self, horizon: int):
        """(X, T): features of states 0 .. n-horizon and their targets log(1 + max of the
        tile's union blocks over that state and the next horizon-1)."""
        import torch
        nsnap = len(self.unions)
        if nsnap < horizon:
            raise ValueError("trace shorter than the horizon")
        trace = torch.stack(self.unions).contiguous()
        ntiles = trace.shape[1]
        targets = torch.empty((nsnap - horizon + 1, ntiles), dtype=torch.float32, device=trace.device)
        vlasov.vl_cost_targets(trace.data_ptr(), nsnap, ntiles, horizon, targets.data_ptr(),
                               torch.cuda.current_stream(trace.device).cuda_stream)
        X = torch.cat(self.features[: nsnap - horizon + 1]).contiguous()
        return X, targets.reshape(-1).contiguous()


def record_run(grid: vlasov.Grid, dt: float, nsteps: int, edge: int = 8, order: str = "xyz",
               form: int = vlasov.VL_FORM_FUSED) -> Trace:
    """Advance `grid` by nsteps, recording the state before each step and after the last."""
    tr = Trace(edge)
    tr.record(grid)
    for _ in range(nsteps):
        grid.translate(dt, order, 1, form)
        tr.record(grid)
    return tr


class CostModel:
    """MLP parameters and Adam moments on the current CUDA device."""

    def __init__(self, seed: int = 0, params=None):
        import torch
        self.torch = torch
        p = inputs.mlp_init(seed) if params is None else np.asarray(params, dtype=np.float32)
        assert p.shape == (vlasov.VL_MLP_NPARAM,)
        self.params = torch.from_numpy(p.copy()).cuda()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self._ws = None

    def _stream(self):
        return self.torch.cuda.current_stream().cuda_stream

    def _workspace(self, n: int):
        need = vlasov.vl_mlp_workspace_bytes(n)
        if self._ws is None or self._ws.numel() < need + 256:
            self._ws = self.torch.empty(need + 256, dtype=self.torch.uint8, device=self.params.device)
        base = self._ws.data_ptr()
        return base + (-base) % 256, need

    def train(self, X, T, epochs: int, lr: float = 3e-3) -> list:
        """Full-batch Adam steps; returns the loss before each step."""
        torch = self.torch
        X = X.contiguous().float()
        T = T.contiguous().float()
        n = X.shape[0]
        ws, nbytes = self._workspace(n)
        losses = torch.zeros(epochs, dtype=torch.float64, device=self.params.device)
        for e in range(epochs):
            self.step += 1
            vlasov.vl_mlp_train_step(self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                     X.data_ptr(), T.data_ptr(), n, self.step, lr, ws, nbytes,
                                     losses[e:].data_ptr(), self._stream())
        return losses.cpu().tolist()

    def predict(self, X):
        torch = self.torch
        X = X.contiguous().float()
        y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        vlasov.vl_mlp_forward(self.params.data_ptr(), X.data_ptr(), X.shape[0], y.data_ptr(), self._stream())
        return y

    def loss(self, X, T) -> float:
        y = self.predict(X)
        return float(((y.double() - T.double()) ** 2).mean())

    def capacity(self, features, margin: float = 0.05) -> int:
        """Pool capacity (blocks) for the next `horizon` steps of the state whose tile
        features are given: (1 + margin) * sum of the predicted tile maxima."""
        n = features.shape[0]
        ws, _ = self._workspace(n)
        need = ((4 * n + 255) // 256) * 256 + 8
        return vlasov.vl_mlp_capacity(self.params.data_ptr(), features.contiguous().data_ptr(), n, margin,
                                      ws, need, self._stream())
