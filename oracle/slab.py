"""The paper's cluster decomposition emulated among CPU ranks (test
infrastructure, like the rest of the oracle).

Sec. 4 runs one RAS domain per GPU: the lattice is cut into x-slabs, every
rank owns one slab of every spinor, the global D needs the neighbouring
slabs' boundary planes (a halo exchange per application), the projection of
Alg. 1 line 4 needs s planes of the residual from each neighbour (with
d = 2s = 0 none), and every dot product of the Krylov solver is a sum over
the ranks.  This module runs that algorithm on torch.distributed ranks (gloo,
CPU) with FP64 numpy arithmetic, taking the per-site operators from the
oracle: the D of a site (``Op.dslash_sites``) and the Dirichlet domain solve
(``Op.domain_solve``).  A rank keeps a full-lattice array per vector but only
its own slab and the planes it has received hold numbers; every other entry
is NaN, so a value that was needed but never sent poisons the result.

Only the tests import this module; the GPU library never does.
"""

from __future__ import annotations

import numpy as np


class SlabRank:
    """One rank of the x-slab decomposition: rank r owns the sites with
    r b <= x < (r + 1) b, b = Lx / world, and its RAS domain is that slab
    extended by s planes on both sides (the oracle's domain r of the blocking
    (b, Ly, Lz, Lt) with extension s)."""

    def __init__(self, op, rank: int, world: int, s: int = 0, n_ras: int = 3, n_dominv: int = 5):
        import torch.distributed as dist
        self.dist = dist
        self.op = op
        self.rank, self.world = rank, world
        L = op.dims
        if L[0] % world:
            raise ValueError("Lx must be divisible by the number of ranks")
        self.b = L[0] // world
        if s > self.b:
            raise ValueError("the extension may not reach past the neighbouring slab")
        self.s, self.n_ras, self.n_dominv = s, n_ras, n_dominv
        self.block = (self.b,) + tuple(L[1:])
        V = op.V
        self.x = np.arange(V) % L[0]
        self.own = (self.x >= rank * self.b) & (self.x < (rank + 1) * self.b)
        self.own_sites = np.nonzero(self.own)[0]
        self.dom_sites, self.dom_bulk = op.domain_sites(self.block, s, rank)
        self.left, self.right = (rank - 1) % world, (rank + 1) % world
        self.dv = 0             # global D applications
        self.halo_bytes = 0     # bytes this rank sent for D halos
        self.proj_bytes = 0     # bytes this rank sent for RAS projections

    # -- communication ----------------------------------------------------
    def _planes(self, xs):
        return np.isin(self.x, np.asarray(xs) % self.op.dims[0])

    def exchange(self, psi, depth: int, count: str):
        """psi with this rank's slab valid -> an array holding also the
        `depth` planes on each side, received from the neighbours; NaN
        elsewhere."""
        import torch
        out = np.full_like(psi, np.nan)
        out[self.own] = psi[self.own]
        if depth == 0:
            return out
        r, b = self.rank, self.b
        lo = self._planes(range(r * b, r * b + depth))             # to the left neighbour
        hi = self._planes(range(r * b + b - depth, r * b + b))     # to the right neighbour
        from_left = self._planes(range(r * b - depth, r * b))
        from_right = self._planes(range(r * b + b, r * b + b + depth))
        send_lo = torch.from_numpy(np.ascontiguousarray(psi[lo]).view(np.float64).copy())
        send_hi = torch.from_numpy(np.ascontiguousarray(psi[hi]).view(np.float64).copy())
        recv_l = torch.empty_like(send_hi)
        recv_r = torch.empty_like(send_lo)
        reqs = [self.dist.isend(send_lo, self.left, tag=0), self.dist.isend(send_hi, self.right, tag=1),
                self.dist.irecv(recv_l, self.left, tag=1), self.dist.irecv(recv_r, self.right, tag=0)]
        for q in reqs:
            q.wait()
        out[from_left] = recv_l.numpy().view(np.complex128).reshape(out[from_left].shape)
        out[from_right] = recv_r.numpy().view(np.complex128).reshape(out[from_right].shape)
        nbytes = send_lo.numel() * 8 + send_hi.numel() * 8
        if count == "halo":
            self.halo_bytes += nbytes
        else:
            self.proj_bytes += nbytes
        return out

    def allsum(self, x: complex) -> complex:
        import torch
        t = torch.tensor([x.real, x.imag], dtype=torch.float64)
        self.dist.all_reduce(t)
        return complex(t[0].item(), t[1].item())

    # -- distributed linear algebra ----------------------------------------
    def local(self):
        """An array for a distributed vector: NaN outside this rank's slab."""
        return np.full(self.op.shape(), np.nan, dtype=np.complex128)

    def D(self, psi):
        """Global D: one halo exchange, then D at this rank's sites."""
        h = self.exchange(psi, 1, "halo")
        out = self.local()
        out[self.own] = self.op.dslash_sites(h, self.own_sites)
        self.dv += 1
        return out

    def dot(self, a, b) -> complex:
        """<a, b> = sum conj(a) b over the lattice (a partial per rank, summed)."""
        return self.allsum(complex(np.vdot(a[self.own], b[self.own])))

    def norm(self, a) -> float:
        return float(np.sqrt(self.dot(a, a).real))

    def ras(self, r):
        """K_RAS r (Alg. 1) with this rank's slab as its domain: the
        projection needs s planes from each neighbour; the domain solve and
        the restriction are local."""
        phi = self.local()
        phi[self.own] = 0
        rho = r.copy()
        for j in range(self.n_ras):
            ext = self.exchange(rho, self.s, "proj")
            rl = ext[self.dom_sites]
            vl = self.op.domain_solve(self.block, self.s, self.rank, rl, n_dominv=self.n_dominv)
            v = self.local()
            v[self.dom_sites[self.dom_bulk]] = vl[self.dom_bulk]
            phi[self.own] += v[self.own]
            if j < self.n_ras - 1:
                rho[self.own] -= self.D(v)[self.own]
        return phi

    def bicgstab(self, b, tol: float, maxit: int, use_ras: bool):
        """Right-preconditioned BiCGStab (van der Vorst, Eq. 3) on the ranks."""
        K = self.ras if use_ras else (lambda y: y.copy())
        x = self.local()
        x[self.own] = 0
        r = b.copy()
        rh = r.copy()
        p = self.local()
        p[self.own] = 0
        v = p.copy()
        rho = alpha = omega = 1.0 + 0j
        bn = self.norm(b)
        it = 0
        while it < maxit:
            rho1 = self.dot(rh, r)
            beta = (rho1 / rho) * (alpha / omega)
            p[self.own] = r[self.own] + beta * (p[self.own] - omega * v[self.own])
            ph = K(p)
            v = self.D(ph)
            rv = self.dot(rh, v)
            if rv == 0:
                break
            alpha = rho1 / rv
            s = self.local()
            s[self.own] = r[self.own] - alpha * v[self.own]
            sh = K(s)
            t = self.D(sh)
            tt = self.dot(t, t).real
            if tt == 0:
                break
            omega = self.dot(t, s) / tt
            x[self.own] += alpha * ph[self.own] + omega * sh[self.own]
            r[self.own] = s[self.own] - omega * t[self.own]
            rho = rho1
            it += 1
            if self.norm(r) <= tol * bn:
                break
        return x, it

    def solve(self, eta, tol: float, inner_tol: float, use_ras: bool = True, max_outer: int = 100):
        """The nested solve with the outer FP64 defect correction (the
        oracle's ora_solve), every vector distributed over the ranks."""
        phi = self.local()
        phi[self.own] = 0
        r = eta.copy()
        en = self.norm(eta)
        outer = inner = 0
        while outer < max_outer:
            rn = self.norm(r)
            if rn <= tol * en:
                break
            rs = self.local()
            rs[self.own] = r[self.own] / rn
            e, it = self.bicgstab(rs, inner_tol, 100000, use_ras)
            inner += it
            outer += 1
            phi[self.own] += rn * e[self.own]
            r[self.own] = eta[self.own] - self.D(phi)[self.own]
        return phi, {"outer_iters": outer, "inner_iters": inner, "dv": self.dv,
                     "true_rel_residual": self.norm(r) / en}
