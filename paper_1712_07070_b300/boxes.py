"""Many independent periodic boxes advanced together on the GPU (marshalling
around amr_hydro_set_box / amr_hydro_advance_boxes only)."""
import numpy as np
import torch

from . import amr_hydro as A


class BoxBatch:
    def __init__(self, gamma=1.4, cfl=0.5, prec=A.AMR_FP32_ACC64, stream=None, device="cuda", scheme=None):
        p = A.make_params(gamma=gamma, cfl=cfl, root_n=(16, 16, 16), prec=prec, **(scheme or {}))
        self.ctx = A.amr_hydro_init(p, stream)
        self.stream = stream
        self.device = torch.device(device)
        self.boxes = []  # (n, [U_a, U_b])

    def close(self):
        if self.ctx is not None:
            A.amr_hydro_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_box(self, U_dense, S_dense=None):
        """Register a periodic n^3 box from its dense state [5][n][n][n]; with
        dual energy also its entropy per unit volume S_dense [n][n][n]."""
        n = U_dense.shape[-1]
        npatch = (n // 8) ** 3
        U = [torch.empty((npatch, 5, 8, 8, 8), dtype=torch.float64, device=self.device) for _ in range(2)]
        d = torch.from_numpy(np.ascontiguousarray(U_dense)).to(self.device)
        A.amr_hydro_pack_uniform(d, n, n, n, U[0], self.stream)
        torch.cuda.synchronize()
        bid = len(self.boxes)
        A.amr_hydro_set_box(self.ctx, bid, n, U[0], U[1])
        S = None
        if S_dense is not None:
            S = [torch.zeros((npatch, 8, 8, 8), dtype=torch.float64, device=self.device) for _ in range(2)]
            tmp = torch.zeros_like(U[0])
            ds = torch.zeros((5, n, n, n), dtype=torch.float64, device=self.device)
            ds[0].copy_(torch.from_numpy(np.ascontiguousarray(S_dense)))
            A.amr_hydro_pack_uniform(ds, n, n, n, tmp, self.stream)
            torch.cuda.synchronize()
            S[0].copy_(tmp[:, 0])
            A.amr_hydro_set_box_entropy(self.ctx, bid, S[0], S[1])
        self.boxes.append((n, U, S))
        return bid

    def advance(self, n_steps, ids=None, log=True):
        ids = list(range(len(self.boxes))) if ids is None else list(ids)
        dt_log = torch.zeros((n_steps, len(ids)), dtype=torch.float64, device=self.device) if log else None
        A.amr_hydro_advance_boxes(self.ctx, ids, n_steps, dt_log)
        return dt_log

    def state(self, i):
        return self.boxes[i][1][A.amr_hydro_box_state(self.ctx, i)]

    def entropy(self, i):
        """The dual-energy entropy field of box i as [n][n][n] (numpy)."""
        n, _, S = self.boxes[i]
        cur = A.amr_hydro_box_state(self.ctx, i)
        tmp = torch.zeros((S[0].shape[0], 5, 8, 8, 8), dtype=torch.float64, device=self.device)
        tmp[:, 0].copy_(S[cur])
        d = torch.empty((5, n, n, n), dtype=torch.float64, device=self.device)
        A.amr_hydro_unpack_uniform(tmp, n, n, n, d, self.stream)
        return d[0].cpu().numpy()

    def download(self, i):
        n = self.boxes[i][0]
        d = torch.empty((5, n, n, n), dtype=torch.float64, device=self.device)
        A.amr_hydro_unpack_uniform(self.state(i), n, n, n, d, self.stream)
        return d.cpu().numpy()

    def tuning(self):
        return A.amr_hydro_box_tuning(self.ctx)
