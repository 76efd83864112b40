"""An AMR hierarchy on the GPU: marshalling around the C ABI only.

torch allocates the caller-owned arrays (root level exactly, levels 1..lmax
with capacity max_patches); regridding, the W-cycle, fix-up, interpolation and
the step all run in libamr_hydro.so.
"""
import numpy as np
import torch

from . import amr_hydro as A


class AmrHierarchy:
    def __init__(self, U_root, lmax, gamma=5.0 / 3.0, cfl=0.5, theta=0.05, nbuf=(8, 4), prec=A.AMR_FP64,
                 max_patches=None, c_inc=0.1, c_dec=0.1, stream=None, device="cuda", regrid_at_start=True, scheme=None,
                 S_root=None, shared_dt=False):
        _, nz, ny, nx = U_root.shape
        self.root = (nx, ny, nz)
        self.lmax = lmax
        self.device = torch.device(device)
        self.stream = stream
        n0 = (nx // 8) * (ny // 8) * (nz // 8)
        if max_patches is None:
            max_patches = 8 * n0
        p = A.make_params(gamma=gamma, cfl=cfl, root_n=(nx, ny, nz), lmax=lmax, prec=prec, **(scheme or {}),
                          max_patches=max(max_patches, n0), theta=theta, c_inc=c_inc, c_dec=c_dec,
                          nbuf=list(nbuf))
        self.ctx = A.amr_hydro_init(p, stream)
        if shared_dt:
            A.amr_hydro_set_shared_dt(self.ctx, True)
        dev = self.device
        corner, sib, parent, child = A.amr_hydro_uniform_tables((nx // 8, ny // 8, nz // 8))
        self.tables = [[torch.from_numpy(a).to(dev) for a in (corner, sib, parent, child)]]
        self.U = [[torch.zeros((n0, 5, 8, 8, 8), dtype=torch.float64, device=dev) for _ in range(2)]]
        dense = torch.from_numpy(np.ascontiguousarray(U_root)).to(dev)
        A.amr_hydro_pack_uniform(dense, nx, ny, nz, self.U[0][0], stream)
        torch.cuda.synchronize()
        A.amr_hydro_set_level(self.ctx, 0, n0, self.U[0][0], self.U[0][1], *self.tables[0], t=0.0)
        # dual energy: the entropy per unit volume of every level, paired with U
        self.S = None
        if S_root is not None:
            self.S = [[torch.zeros((n0, 8, 8, 8), dtype=torch.float64, device=dev) for _ in range(2)]]
            tmp = torch.zeros_like(self.U[0][0])
            ds = torch.zeros((5, nz, ny, nx), dtype=torch.float64, device=dev)
            ds[0].copy_(torch.from_numpy(np.ascontiguousarray(S_root)))
            A.amr_hydro_pack_uniform(ds, nx, ny, nz, tmp, stream)
            torch.cuda.synchronize()
            self.S[0][0].copy_(tmp[:, 0])
            A.amr_hydro_set_entropy(self.ctx, 0, self.S[0][0], self.S[0][1])
        mp = p.max_patches
        for l in range(1, lmax + 1):
            U = [torch.zeros((mp, 5, 8, 8, 8), dtype=torch.float64, device=dev) for _ in range(2)]
            t = [torch.full((mp, 3), -1, dtype=torch.int32, device=dev),
                 torch.full((mp, 26), -1, dtype=torch.int32, device=dev),
                 torch.full((mp,), -1, dtype=torch.int32, device=dev),
                 torch.full((mp,), -1, dtype=torch.int32, device=dev)]
            self.U.append(U)
            self.tables.append(t)
            A.amr_hydro_bind_level(self.ctx, l, U[0], U[1], *t)
            if self.S is not None:
                S = [torch.zeros((mp, 8, 8, 8), dtype=torch.float64, device=dev) for _ in range(2)]
                self.S.append(S)
                A.amr_hydro_set_entropy(self.ctx, l, S[0], S[1])
        if regrid_at_start:
            for l in range(lmax):
                A.amr_hydro_regrid(self.ctx, l)

    def close(self):
        if self.ctx is not None:
            A.amr_hydro_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n_patches(self, l):
        return A.amr_hydro_level_info(self.ctx, l)[0]

    def state(self, l):
        n = self.n_patches(l)
        cur, _, _ = A.amr_hydro_get_state(self.ctx, l)
        return self.U[l][cur][:n]

    def set_gravity(self, G, omega=1.7, iters=60, acc_order=2):
        """Self-gravity in the W-cycle from now on (solves every level's potential)."""
        A.amr_hydro_set_gravity(self.ctx, G, omega, iters, acc_order)

    def gravity(self, l):
        """Level l's newest potential [n][8][8][8] and acceleration [n][3][8][8][8]."""
        n = self.n_patches(l)
        phi = torch.zeros((n, 8, 8, 8), dtype=torch.float64, device=self.device)
        acc = torch.zeros((n, 3, 8, 8, 8), dtype=torch.float64, device=self.device)
        A.amr_hydro_level_gravity(self.ctx, l, phi, acc)
        return phi, acc

    def entropy(self, l):
        """Dual energy: level l's current entropy per unit volume, [n_patches][8][8][8]."""
        n = self.n_patches(l)
        cur, _, _ = A.amr_hydro_get_state(self.ctx, l)
        return self.S[l][cur][:n]

    def time(self, l):
        return A.amr_hydro_get_state(self.ctx, l)[1]

    def corners(self, l):
        return self.tables[l][0][:self.n_patches(l)].cpu().numpy()

    def advance_root(self, dt0=-1.0):
        return A.amr_hydro_advance_root(self.ctx, dt0)

    def conserved_total(self):
        tot = np.zeros(5)
        for l in range(self.lmax + 1):
            if self.n_patches(l):
                tot += np.array(A.amr_hydro_conserved_sum(self.ctx, l))
        return tot
