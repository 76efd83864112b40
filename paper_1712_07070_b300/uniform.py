"""Uniform periodic grids (one fully covered AMR level) on the GPU.

Marshalling around the C ABI only: torch allocates the caller-owned device
arrays; packing, stepping, reductions all run in libamr_hydro.so.
"""
import numpy as np
import torch

from . import amr_hydro as A


class UniformGrid:
    """A periodic nx x ny x nz box (multiples of 16) as one level of 8^3 patches."""

    def __init__(self, shape, gamma=5.0 / 3.0, cfl=0.5, prec=A.AMR_FP64, box_x=1.0, stream=None,
                 device="cuda", scheme=None):
        """scheme: optional dict of make_params' scheme options (limiter, riemann, minmod_coeff,
        scheme, recon, fallback, dt_min)."""
        nx, ny, nz = shape
        self.shape = (nx, ny, nz)
        self.device = torch.device(device)
        self.stream = stream
        p = A.make_params(gamma=gamma, cfl=cfl, root_n=(nx, ny, nz), **(scheme or {}),
                          box=(box_x, box_x * ny / nx, box_x * nz / nx), prec=prec)
        self.params = p
        self.dh = box_x / nx
        self.ctx = A.amr_hydro_init(p, stream)
        npch = (nx // 8, ny // 8, nz // 8)
        self.n_patches = npch[0] * npch[1] * npch[2]
        corner, sib, parent, child = A.amr_hydro_uniform_tables(npch)
        self.tables = [torch.from_numpy(a).to(self.device) for a in (corner, sib, parent, child)]
        self._stage = None
        self.U = [torch.zeros((self.n_patches, 5, 8, 8, 8), dtype=torch.float64, device=self.device)
                  for _ in range(2)]
        A.amr_hydro_set_level(self.ctx, 0, self.n_patches, self.U[0], self.U[1], *self.tables, t=0.0)

    def close(self):
        if self.ctx is not None:
            A.amr_hydro_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def state(self):
        cur, _, _ = A.amr_hydro_get_state(self.ctx, 0)
        return self.U[cur]

    def time(self):
        _, t, _ = A.amr_hydro_get_state(self.ctx, 0)
        return t

    def _staging(self):
        if self._stage is None:
            nx, ny, nz = self.shape
            self._stage = torch.empty((5, nz, ny, nx), dtype=torch.float64, device=self.device)
        return self._stage

    def _torch_stream(self):
        if self.stream is None:
            return torch.cuda.default_stream(self.device)
        return torch.cuda.ExternalStream(self.stream, device=self.device)

    def upload(self, U_dense):
        """U_dense: [5][nz][ny][nx] float64 (numpy, host or device tensor) ->
        the current state (copy into a device staging buffer, pack kernel)."""
        d = torch.from_numpy(np.ascontiguousarray(U_dense)) if isinstance(U_dense, np.ndarray) else U_dense
        st = self._staging()
        with torch.cuda.stream(self._torch_stream()):
            st.copy_(d, non_blocking=d.device.type == "cpu" and d.is_pinned())
            nx, ny, nz = self.shape
            A.amr_hydro_pack_uniform(st, nx, ny, nz, self.state(), self.stream)
        A.amr_hydro_touch_level(self.ctx, 0)

    def download(self, out=None):
        """Current state as [5][nz][ny][nx]: a numpy array, or copied into
        ``out`` (a host or device tensor; asynchronous for pinned host)."""
        nx, ny, nz = self.shape
        st = self._staging()
        with torch.cuda.stream(self._torch_stream()):
            A.amr_hydro_unpack_uniform(self.state(), nx, ny, nz, st, self.stream)
            if out is None:
                return st.cpu().numpy()
            out.copy_(st, non_blocking=out.device.type == "cpu" and out.is_pinned())
            return out

    def set_entropy(self, S_dense):
        """Dual energy: the entropy per unit volume s = P / rho^(gamma-1) of the
        current state, [nz][ny][nx] float64; allocates the two entropy slot
        buffers and registers them (params.dual_energy)."""
        cur, _, _ = A.amr_hydro_get_state(self.ctx, 0)
        self.S = [torch.zeros((self.n_patches, 8, 8, 8), dtype=torch.float64, device=self.device)
                  for _ in range(2)]
        A.amr_hydro_set_entropy(self.ctx, 0, self.S[cur], self.S[1 - cur])
        tmp = torch.zeros_like(self.U[0])
        st = self._staging()
        nx, ny, nz = self.shape
        with torch.cuda.stream(self._torch_stream()):
            st.zero_()
            st[0].copy_(torch.as_tensor(np.ascontiguousarray(S_dense)))
            A.amr_hydro_pack_uniform(st, nx, ny, nz, tmp, self.stream)
            self.S[cur].copy_(tmp[:, 0])
        torch.cuda.synchronize(self.device)

    def entropy(self):
        """The current entropy field as [nz][ny][nx] (numpy)."""
        cur, _, _ = A.amr_hydro_get_state(self.ctx, 0)
        tmp = torch.zeros_like(self.U[0])
        st = self._staging()
        nx, ny, nz = self.shape
        with torch.cuda.stream(self._torch_stream()):
            tmp[:, 0].copy_(self.S[cur])
            A.amr_hydro_unpack_uniform(tmp, nx, ny, nz, st, self.stream)
            return st[0].cpu().numpy()

    def gravity(self, G, order=2):
        """The FFT potential and acceleration of the current density:
        ([n_patches][8][8][8], [n_patches][3][8][8][8]) device tensors."""
        phi = torch.zeros((self.n_patches, 8, 8, 8), dtype=torch.float64, device=self.device)
        acc = torch.zeros((self.n_patches, 3, 8, 8, 8), dtype=torch.float64, device=self.device)
        A.amr_hydro_poisson_root(self.ctx, G, phi, acc, order)
        return phi, acc

    def step_gravity(self, G, acc_n, dt=-1.0, order=2, c_acc=0.0):
        """One hydro step coupled to self-gravity (predictor with acc_n, the
        acceleration of the current state; the potential of the predicted
        density; the corrector); dt < 0 with c_acc > 0 also obeys Eq. (acc).
        Returns (phi, acc) of the new state."""
        phi = torch.zeros((self.n_patches, 8, 8, 8), dtype=torch.float64, device=self.device)
        acc = torch.zeros((self.n_patches, 3, 8, 8, 8), dtype=torch.float64, device=self.device)
        A.amr_hydro_advance_gravity(self.ctx, dt, G, acc_n, phi, acc, order, c_acc)
        return phi, acc

    def to_dense(self, slots):
        """Patch-slot arrays [n_patches][...][8][8][8] -> [...][nz][ny][nx] (numpy)."""
        a = slots.cpu().numpy() if isinstance(slots, torch.Tensor) else slots
        nx, ny, nz = self.shape
        out = np.zeros(a.shape[1:-3] + (nz, ny, nx))
        for s, (x, y, z) in enumerate(self.tables[0].cpu().numpy()):
            out[..., z:z + 8, y:y + 8, x:x + 8] = a[s]
        return out

    def min_dt(self):
        return A.amr_hydro_min_dt(self.ctx, 0)

    def step(self, dt=-1.0, count_unphysical=False):
        return A.amr_hydro_advance_level(self.ctx, 0, dt, count_unphysical)

    def step_host(self, U_in, U_out, dt=-1.0):
        """One step from host state U_in to host state U_out ([5][nz][ny][nx]
        float64 tensors or arrays on the host; page-locked memory lets the
        copies overlap the update).  Returns the CFL dt of U_out, the dt to
        pass to the next call of a chained run."""
        return A.amr_hydro_advance_host(self.ctx, U_in, U_out, dt)
