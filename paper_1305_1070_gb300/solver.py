"""One pass of the GPU path for a device workload: contact self-energies (S1a),
lesser/greater self-energies, assembly and fold (S1-S3), selected inversion for
G^r, G^< and G^> (S4-S8), all through the C ABI of ``include/ndgf.h``.

torch is used for device memory and streams only; every arithmetic step runs
in the library's CUDA kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ndgf


RESID_MAX = 1e-6    # backward error above which an energy is recomputed (the density gate's 1e-6)
GROWTH_MAX = 1e4    # fold growth max|Psi| that alone triggers a recomputation


def certificate_flags(cert, resid_max: float = RESID_MAX, growth_max: float = GROWTH_MAX):
    """Energies whose S9 certificate ([n_e, 8], nd_certificate) fails: a
    relative FP64 residual of the diagonal of A G^r = I or of
    A G^< = Sigma^< G^a (entries 6, 7: backward errors) above resid_max, a fold
    growth max|Psi| above growth_max, a stored entry not found, or a non-finite
    value.  The default backward-error threshold is the metric's density
    tolerance: measured, the delayed-pivot paths stay below 3.3e-9 on the
    superlattice, failed plain eliminations are above 1.3e-5, and on the
    nanotube 62 of 1,024 energies (those next to the lead's edge-state pole)
    exceed it; growth alone (up to 1.1e3 on the nanotube, whose backward errors
    mostly stay small) is flagged only when extreme."""
    bad = (cert[:, 6] > resid_max) | (cert[:, 7] > resid_max) | (cert[:, 4] > growth_max) | (cert[:, 5] > 0)
    return bad | ~torch.isfinite(cert).all(dim=1)


class Solver:
    def __init__(self, dev, tr, *, precision: int = ndgf.ND_PREC_FP64, max_ne: int | None = None,
                 leaf_size: int = 64, split_permille: int = 0, delay: int = 0, tile: str = "auto",
                 adjoint: bool = False, graph: bool = False, device: str = "cuda"):
        self.dev, self.tr = dev, tr
        # a complex H (or lead) is rejected before anything is allocated
        ndgf.require_real(dev.values, "Solver: H values")
        for lead in dev.leads:
            for block in ("H00", "H01", "tau"):
                ndgf.require_real(getattr(lead, block), f"Solver: lead {block}")
        self.device = torch.device(device)
        self.n = dev.n
        cp = np.concatenate([[0], np.cumsum([len(c) for c in dev.contacts])]).astype(np.int32)
        ci = np.concatenate(dev.contacts).astype(np.int32) if dev.contacts else np.zeros(0, np.int32)
        self.plan = ndgf.nd_analyze(dev.n, dev.rowptr, dev.colind, cp, ci, dev.coords, leaf_size, split_permille,
                                    delay=delay)
        self.info = ndgf.nd_plan_query(self.plan)
        self.m_c = [len(c) for c in dev.contacts]
        self.off = np.concatenate([[0], np.cumsum([m * m for m in self.m_c])]).astype(np.int64)
        self.sigma_elems = int(self.off[-1])
        self.max_ne = int(max_ne or tr.n_e)
        self.precision = precision
        flags = ndgf.ND_FACT_PHONON if tr.gamma_ph > 0.0 else 0
        flags |= {"auto": 0, "large": ndgf.ND_FACT_TILE_LARGE, "small": ndgf.ND_FACT_TILE_SMALL,
                  "xl": ndgf.ND_FACT_TILE_XL, "tc": ndgf.ND_FACT_GEMM_TC, "alu": ndgf.ND_FACT_GEMM_ALU}[tile]
        if adjoint:
            flags |= ndgf.ND_FACT_ADJOINT
        if graph:
            flags |= ndgf.ND_FACT_GRAPH
        self.fact = ndgf.nd_fact_create(self.plan, self.max_ne, precision, flags)
        self.leads = [ndgf.nd_lead_create(l.H00, l.H01, l.tau) for l in dev.leads]
        kw = dict(device=self.device)
        self.H = torch.as_tensor(dev.values, dtype=torch.float64, **kw).contiguous()
        self.H0 = self.H.clone()
        # CSR position of every diagonal entry (onsite potentials enter there)
        diag = np.full(dev.n, -1, dtype=np.int64)
        for r in range(dev.n):
            row = dev.colind[dev.rowptr[r]:dev.rowptr[r + 1]]
            hit = np.nonzero(row == r)[0]
            if hit.size:
                diag[r] = dev.rowptr[r] + hit[0]
        self.diag_pos = torch.as_tensor(diag, **kw)
        self.E = torch.zeros(self.max_ne, dtype=torch.float64, **kw)
        se = max(1, self.sigma_elems)
        self.sig_r = torch.zeros(self.max_ne, se, dtype=torch.complex128, **kw)
        self.sig_l = torch.zeros_like(self.sig_r)
        self.sig_g = torch.zeros_like(self.sig_r)
        self.ph = tr.gamma_ph > 0.0
        if self.ph:
            self.ph_r = torch.zeros(self.max_ne, self.n, dtype=torch.complex128, **kw)
            self.ph_l = torch.zeros_like(self.ph_r)
            self.ph_g = torch.zeros_like(self.ph_r)
        else:
            self.ph_r = self.ph_l = self.ph_g = None
        self.Gr = torch.zeros(self.max_ne, self.n, dtype=torch.complex128, **kw)
        self.Gl = torch.zeros_like(self.Gr)
        self.Gg = torch.zeros_like(self.Gr)

    def step(self, energies, lesser: bool = True):
        """Diagonals of G^r, G^<, G^> (caller order) for the given energies."""
        n_e = len(energies)
        if n_e > self.max_ne:
            raise ValueError("more energies than the workspace holds")
        E = self.E[:n_e]
        if isinstance(energies, torch.Tensor):
            E.copy_(energies)
        else:
            E.copy_(torch.as_tensor(np.asarray(energies, dtype=np.float64)))
        self._self_energies(n_e)
        return self._solve(n_e, lesser)

    def _self_energies(self, n_e: int):
        """Contact, lesser/greater and phonon self-energies of self.E[:n_e] (S1a)."""
        E = self.E[:n_e]
        tr = self.tr
        for c, lead in enumerate(self.leads):
            ndgf.nd_lead_sigma(lead, E, n_e, tr.eta, self.sig_r, self.sigma_elems, int(self.off[c]))
        if self.leads:
            # Fermi level per contact: the pattern of tr.mu repeats over the devices of a union
            mu = [tr.mu[c % len(tr.mu)] for c in range(len(self.m_c))]
            ndgf.nd_sigma_lesser_fermi(self.sig_r, n_e, self.m_c, mu, tr.kT, E, self.sig_l, self.sig_g)
        if self.ph:
            mu_ph = tr.mu_ph if tr.mu_ph is not None else 0.5 * (tr.mu[0] + tr.mu[1])
            ndgf.nd_phonon_const(self.n, n_e, tr.gamma_ph, mu_ph, tr.kT, E, self.ph_r, self.ph_l, self.ph_g)

    def step_host(self, E_host, Gr_host, Gl_host, Gg_host, H_host=None):
        """step() through the library's host-buffer path: the energies (and H,
        when given) are host arrays that nd_factor stages to the device, and
        nd_diag_green writes the three diagonals ([n_e, n] complex128) straight
        into the host arrays Gr_host, Gl_host, Gg_host (pinned memory keeps the
        copies asynchronous).  The lead self-energies are computed on the device
        from a device copy of the energies."""
        n_e = len(E_host)
        if n_e > self.max_ne:
            raise ValueError("more energies than the workspace holds")
        self.E[:n_e].copy_(torch.as_tensor(E_host), non_blocking=True)
        self._self_energies(n_e)
        ndgf.nd_factor(self.fact, self.H if H_host is None else H_host, self.sig_r if self.leads else None, self.ph_r,
                       E_host, n_e, self.tr.eta)
        ndgf.nd_diag_green(self.fact, self.sig_l, self.sig_g, self.ph_l, self.ph_g, Gr_host, Gl_host, Gg_host)

    def set_potential(self, U):
        """On-site potential energy U ([n] real, eV, caller order) for the following
        steps: it enters nd_factor as a real diagonal self-energy term, so that
        A = (E + i eta) I - H - diag(U) - Sigma (H stays untouched)."""
        if self.ph:
            raise ValueError("set_potential with a phonon self-energy is not supported")
        if not hasattr(self, "pot"):
            self.pot = torch.zeros(self.max_ne, self.n, dtype=torch.complex128, device=self.device)
        self.pot.real.copy_(torch.as_tensor(U, dtype=torch.float64, device=self.device).expand(self.max_ne, self.n))

    def _solve(self, n_e: int, lesser: bool = True):
        """Fold and diagonals for the energies, contact and phonon self-energies in place."""
        E = self.E[:n_e]
        diag = self.ph_r if self.ph else getattr(self, "pot", None)
        ndgf.nd_factor(self.fact, self.H, self.sig_r if self.leads else None, diag, E, n_e, self.tr.eta)
        ndgf.nd_diag_green(self.fact, self.sig_l if lesser else None, self.sig_g if lesser else None,
                           self.ph_l if lesser else None, self.ph_g if lesser else None,
                           self.Gr, self.Gl if lesser else None, self.Gg if lesser else None)
        return self.Gr[:n_e], self.Gl[:n_e], self.Gg[:n_e]

    def autotune(self, energies, reps: int = 1) -> dict:
        """nd_autotune on these energies (at most max_ne): each GEMM launch of
        the fold and the extraction takes the kernel measured fastest on this
        workload for all later steps.  Returns the tuning summary."""
        n_e = len(energies)
        E = self.E[:n_e]
        E.copy_(energies if isinstance(energies, torch.Tensor) else torch.as_tensor(np.asarray(energies, dtype=np.float64)))
        self._self_energies(n_e)
        return ndgf.nd_autotune(self.fact, self.H, self.sig_r if self.leads else None, self.ph_r, self.sig_l,
                                self.sig_g, self.ph_l, self.ph_g, E, n_e, self.tr.eta, reps)

    def choice(self) -> np.ndarray:
        """The kernel of every step (nd_fact_get_choice), to store a tuning."""
        return ndgf.nd_fact_get_choice(self.fact)

    def set_choice(self, choice) -> None:
        """Apply a stored kernel choice (nd_fact_set_choice), e.g. one tuned on
        a handle of the same plan with more energies."""
        ndgf.nd_fact_set_choice(self.fact, choice)

    def scba(self, energies, D: float, *, mix: float = 1.0, updates: int | None = None, tol: float = 1e-13,
             max_updates: int = 2000):
        """Self-consistent Born iteration of an elastic local phonon self-energy,
        Sigma_ph,jj = D G_jj for r, <, > (D in eV^2; nd_phonon_scba), starting from
        the constant broadening of the transport parameters (gamma_ph > 0: it also
        reserves the phonon workspace).  Each update is followed by a solve; the
        loop stops after `updates` updates, or when the relative change of the
        self-energies falls to `tol`.  Returns (Gr, Gl, Gg, updates, last change)."""
        if not self.ph:
            raise ValueError("scba needs gamma_ph > 0 (phonon workspace and first iterate)")
        n_e = len(energies)
        self.step(energies)
        stats = torch.zeros(2, dtype=torch.float64, device=self.device)
        n_upd, change = 0, float("inf")
        limit = updates if updates is not None else max_updates
        while n_upd < limit:
            ndgf.nd_phonon_scba(self.n, n_e, D, mix, self.Gr, self.Gl, self.Gg, self.ph_r, self.ph_l, self.ph_g,
                                stats)
            self._solve(n_e)
            n_upd += 1
            st = stats.cpu().numpy()
            change = float(st[0] / st[1]) if st[1] > 0 else float(st[0])
            if updates is None and change <= tol:
                break
        return self.Gr[:n_e], self.Gl[:n_e], self.Gg[:n_e], n_upd, change

    def certificate(self, n_e: int):
        """Per-energy certificate of the last step: [n_e, 8] = (max|A G - I|_jj,
        max|G_jj|, max|A G^< - Sigma^< G^a|_jj, max|G^<_jj|, max|Psi|, entries
        not found, and the two residuals relative to their terms)."""
        cert = torch.zeros(n_e, 8, dtype=torch.float64, device=self.device)
        ndgf.nd_certificate(self.fact, cert)
        return cert

    def step_certified(self, energies, fallback: "Solver", *, resid_max: float = RESID_MAX,
                       growth_max: float = GROWTH_MAX):
        """step() followed by the S9 certificate: energies whose relative FP64
        residual of diag(A G^r - I) or diag(A G^< - Sigma^< G^a) exceeds
        resid_max, or whose fold growth max|Psi| exceeds growth_max, are
        recomputed by `fallback` (a complex128 Solver of the same device) and
        their rows overwritten.  Returns (Gr, Gl, Gg, cert, redone) with cert the
        [n_e, 8] certificate of this solver's pass and redone the indices of the
        recomputed energies (a device tensor)."""
        n_e = len(energies)
        E = energies if isinstance(energies, torch.Tensor) else torch.as_tensor(
            np.asarray(energies, dtype=np.float64), device=self.device)
        Gr, Gl, Gg = self.step(E)
        cert = self.certificate(n_e)
        idx = torch.nonzero(certificate_flags(cert, resid_max, growth_max)).flatten()
        k = int(idx.numel())
        for c0 in range(0, k, fallback.max_ne):
            sel = idx[c0:c0 + fallback.max_ne]
            r, l, g = fallback.step(E[sel])
            Gr[sel], Gl[sel], Gg[sel] = r, l, g
        return Gr, Gl, Gg, cert, idx

    def singular_pivots(self) -> int:
        return ndgf.nd_fact_status(self.fact)

    def current(self, contact: int, n_e: int):
        """Terminal current spectrum i_c(E) = Tr[Sigma^<_c G^>_cc - Sigma^>_c G^<_cc] of the last step
        (real and imaginary parts, the latter zero up to rounding)."""
        re = torch.zeros(n_e, dtype=torch.float64, device=self.device)
        im = torch.zeros(n_e, dtype=torch.float64, device=self.device)
        ndgf.nd_contact_current(self.fact, contact, re, im)
        return re, im

    def set_onsite(self, V):
        """H = H0 + diag(V) for the following steps (V: [n] float64, caller order)."""
        if bool((self.diag_pos < 0).any()):
            raise ValueError("the pattern of H lacks diagonal entries")
        self.H.copy_(self.H0)
        self.H.index_add_(0, self.diag_pos, torch.as_tensor(V, dtype=torch.float64, device=self.device))

    def density_gradient_terms(self, c, n_e: int):
        """t[e][k] of the last step for the weights c (see nd_density_gradient):
        d(sum_j c_j n_j)/dV_k = (2/pi) sum_e w_e Im t[e][k]."""
        t = torch.zeros(n_e, self.n, dtype=torch.complex128, device=self.device)
        ndgf.nd_density_gradient(self.fact, torch.as_tensor(c, dtype=torch.float64, device=self.device).contiguous(), t)
        return t

    def lead_status(self):
        """Per lead (n_unconverged, n_singular) of the decimation since the last query."""
        return [ndgf.nd_lead_status(lead) for lead in self.leads]

