"""Self-consistent Schroedinger-Poisson iteration on the GPU path (the paper
motivates the diagonal of G^< by the electron density that feeds Poisson's
equation, Sec. 1; the electrostatics are not in the paper).

Unknown: the electrostatic potential energy U (eV) of the device sites, which
enters A as a real diagonal term: A = (E + i eta) I - H - diag(U) - Sigma.
With the Poisson operator K of nd_poisson (Dirichlet at the transport ends,
Neumann at the edges), the coupling lam (eV per electron) and a background
charge nD (electrons per site):
    F(U) = K U - lam (n(U) - nD) = 0,       J(U) = K - lam dn/dU.
Each Newton step solves J z = -F by GMRES, right-preconditioned by the
screened operator M = K + lam D (D_j = -((dn/dU) 1)_j, the local response of
the density to a uniform potential; M^{-1} by conjugate gradients
preconditioned with the direct solve of K + shift I), with the products dn/dU v from
nd_density_jvp (the stored factorization of every energy chunk is reused
across the GMRES iterations), and updates U <- U + a z, a = 1 unless halving
it is needed for |F| to decrease.  Every vector operation runs in the library
(nd_vec_dot, nd_vec_axpby, nd_poisson_*); torch supplies device memory, the
host keeps only the small Hessenberg least-squares problem of GMRES.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import ndgf
from .solver import Solver


class SchrodingerPoisson:
    def __init__(self, dev, tr, L: int, W: int, lam: float, nD, *, precision: int = ndgf.ND_PREC_FP64,
                 delay: int = 2, leaf_size: int = 16, chunk: int | None = None, gmres_tol: float = 1e-12,
                 gmres_max: int = 40):
        if dev.n != L * W:
            raise ValueError("the device must be the L x W grid")
        self.n, self.L, self.W, self.lam = dev.n, L, W, float(lam)
        self.gmres_tol, self.gmres_max = gmres_tol, gmres_max
        E = np.asarray(tr.energies, dtype=np.float64)
        chunk = chunk or len(E)
        self.parts = []
        d = np.diff(E)
        w = np.zeros(len(E))
        w[:-1] += 0.5 * d
        w[1:] += 0.5 * d
        for c0 in range(0, len(E), chunk):
            s = Solver(dev, tr, precision=precision, max_ne=min(chunk, len(E) - c0), delay=delay,
                       leaf_size=leaf_size, adjoint=True)
            Ec = torch.as_tensor(E[c0:c0 + chunk], device="cuda")
            wc = torch.as_tensor(w[c0:c0 + chunk], device="cuda")
            t = torch.zeros(len(Ec), dev.n, dtype=torch.complex128, device="cuda")
            self.parts.append((s, Ec, wc, t))
        self.P = ndgf.nd_poisson_create(L, W)
        z = lambda: torch.zeros(dev.n, dtype=torch.float64, device="cuda")
        self.nD = torch.as_tensor(np.asarray(nD, dtype=np.float64), device="cuda").expand(dev.n).contiguous()
        self.U, self.F, self.dens, self._tmp, self._tmp2 = z(), z(), z(), z(), z()
        self._dot = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.shift = 0.0
        self.D, self._w1 = z(), z()
        self._c = [z() for _ in range(4)]

    # ---- library vector operations
    def dot(self, x, y) -> float:
        ndgf.nd_vec_dot(x, y, self.n, self._dot)
        return float(self._dot.item())

    def axpby(self, a, x, b, y):
        ndgf.nd_vec_axpby(a, x, b, y, self.n)

    # ---- the maps
    def density(self, U, out):
        """n(U) into out; leaves every chunk's factorization of H + diag(U) in place."""
        for k, (s, Ec, wc, _) in enumerate(self.parts):
            s.set_potential(U)
            s.step(Ec)
            ndgf.nd_fact_density(s.fact, wc, 1.0 / math.pi, 1 if k else 0, out)
        return out

    def residual(self, U, out):
        """F(U) = K U - lam (n(U) - nD) into out (and the density into self.dens)."""
        self.density(U, self.dens)
        ndgf.nd_poisson_apply(self.P, U, out)
        self.axpby(-self.lam, self.dens, 1.0, out)
        self.axpby(self.lam, self.nD, 1.0, out)
        return out

    def jvp(self, v, out):
        """(dn/dU) v into out, on the factorizations of the last density() call."""
        for k, (s, Ec, wc, t) in enumerate(self.parts):
            ndgf.nd_density_jvp(s.fact, v, t)
            ndgf.nd_density(t, wc, len(Ec), self.n, 2.0 / math.pi, 1 if k else 0, out)
        return out

    def _op(self, y, out):
        """(J M^{-1}) y: J z = K z - lam (dn/dU) z for z = M^{-1} y."""
        self.precondition(y, self._tmp)
        self.jvp(self._tmp, out)
        ndgf.nd_poisson_apply(self.P, self._tmp, self._tmp2)
        self.axpby(1.0, self._tmp2, -self.lam, out)
        return out

    def screening(self):
        """The preconditioner M = K + lam D of the next Newton step, D_j =
        max(0, -((dn/dU) 1)_j): the local response of the density to a uniform
        potential (a Thomas-Fermi screening of K, large in the wells, near zero
        in the barriers), at the factorizations of the last density() call.
        Also sets the uniform shift lam mean(D) of the inner preconditioner."""
        ones = torch.ones(self.n, dtype=torch.float64, device="cuda")
        self.jvp(ones, self._w1)
        ndgf.nd_vec_scale_pos(-self.lam, self._w1, self.D, self.n)
        self.shift = self.dot(self.D, ones) / self.n

    def _mapply(self, u, out):
        ndgf.nd_poisson_apply(self.P, u, out)
        ndgf.nd_vec_mul(self.D, u, self._w1, self.n)
        self.axpby(1.0, self._w1, 1.0, out)

    def precondition(self, r, z):
        """z = M^{-1} r by conjugate gradients on the SPD M = K + lam D,
        preconditioned by the direct solve of K + shift I, to a relative
        residual of 1e-12 (so that M stays the same operator for GMRES)."""
        rr, p, q, y = self._c[0], self._c[1], self._c[2], self._c[3]
        z.zero_()
        rr.copy_(r)
        bn = math.sqrt(self.dot(r, r))
        if bn == 0.0:
            return z
        ndgf.nd_poisson_solve(self.P, rr, y, shift=self.shift)
        p.copy_(y)
        rho = self.dot(rr, y)
        for _ in range(500):
            self._mapply(p, q)
            alpha = rho / self.dot(p, q)
            self.axpby(alpha, p, 1.0, z)
            self.axpby(-alpha, q, 1.0, rr)
            if math.sqrt(self.dot(rr, rr)) <= 1e-12 * bn:
                break
            ndgf.nd_poisson_solve(self.P, rr, y, shift=self.shift)
            rho_new = self.dot(rr, y)
            self.axpby(1.0, y, rho_new / rho, p)
            rho = rho_new
        return z

    def gmres(self, b):
        """z with J z = b (right preconditioning by K^{-1}); returns (z, iterations, relative residual)."""
        n, m = self.n, self.gmres_max
        beta = math.sqrt(self.dot(b, b))
        z = torch.zeros(n, dtype=torch.float64, device="cuda")
        if beta == 0.0:
            return z, 0, 0.0
        V = [torch.zeros(n, dtype=torch.float64, device="cuda")]
        self.axpby(1.0 / beta, b, 0.0, V[0])
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        rel = 1.0
        for j in range(m):
            w = torch.zeros(n, dtype=torch.float64, device="cuda")
            self._op(V[j], w)
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = self.dot(w, V[i])
                self.axpby(-H[i, j], V[i], 1.0, w)
            hn = math.sqrt(self.dot(w, w))
            H[j + 1, j] = hn
            for i in range(j):  # the earlier Givens rotations
                a, c = H[i, j], H[i + 1, j]
                H[i, j], H[i + 1, j] = cs[i] * a + sn[i] * c, -sn[i] * a + cs[i] * c
            r = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = (H[j, j] / r, H[j + 1, j] / r) if r > 0 else (1.0, 0.0)
            H[j, j], H[j + 1, j] = r, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            rel = abs(g[j + 1]) / beta
            if rel <= self.gmres_tol or hn == 0.0:
                break
            nxt = torch.zeros(n, dtype=torch.float64, device="cuda")
            self.axpby(1.0 / hn, w, 0.0, nxt)
            V.append(nxt)
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        acc = torch.zeros(n, dtype=torch.float64, device="cuda")
        for i in range(k):
            self.axpby(float(y[i]), V[i], 1.0, acc)
        self.precondition(acc, z)
        return z, k, rel

    def newton(self, steps: int, U0=None, max_halvings: int = 5):
        """Runs `steps` Newton steps from U0 (default 0).  Each step: the
        screening shift of the preconditioner, GMRES for J z = -F, then U + a z
        with a = 1, 1/2, ... until |F| decreases (at most max_halvings
        halvings; the full step is taken whenever it decreases |F|).  Returns
        the iterates (host [steps + 1, n]), the 2-norms |F| of each iterate,
        the GMRES iteration counts and the step lengths a."""
        if U0 is not None:
            self.U.copy_(torch.as_tensor(np.asarray(U0, dtype=np.float64), device="cuda"))
        else:
            self.U.zero_()
        its, res, kry, lens = [self.U.cpu().numpy()], [], [], []
        b = torch.zeros(self.n, dtype=torch.float64, device="cuda")
        Ut = torch.zeros_like(self.U)
        Ft = torch.zeros_like(self.U)
        self.residual(self.U, self.F)
        fn = math.sqrt(self.dot(self.F, self.F))
        for _ in range(steps):
            res.append(fn)
            self.screening()
            self.axpby(-1.0, self.F, 0.0, b)
            z, k, _ = self.gmres(b)
            kry.append(k)
            a = 1.0
            for h in range(max_halvings + 1):
                Ut.copy_(self.U)
                self.axpby(a, z, 1.0, Ut)
                self.residual(Ut, Ft)  # leaves the factorizations at Ut
                ft = math.sqrt(self.dot(Ft, Ft))
                if ft < (1.0 - 1e-4 * a) * fn or h == max_halvings:
                    break
                a *= 0.5
            lens.append(a)
            self.U.copy_(Ut)
            self.F.copy_(Ft)
            fn = ft
            its.append(self.U.cpu().numpy())
        res.append(fn)
        return np.array(its), np.array(res), kry, lens
