"""Planted mistakes in the oracle, each caught by at least one pin.

Every oracle module is pinned by tests against something other than itself
(test_oracle_*.py).  Here each module's source is changed in memory by one
plausible mistake -- a dropped term, a wrong sign, a transposed operand, a
swapped index or occupation, a copy-paste slip -- the changed functions
replace the originals wherever the oracle and the pin modules hold them, and
the pins of that module run: at least one must fail.  A control run per module
(no change) shows that the harness alone fails nothing.  The source files are
never written.

Mistakes that cannot change any result on the pinned inputs are not listed:
for example a transpose in place of a conjugate transpose of a matrix that is
real symmetric on every workload (the lead coupling of a square lattice)."""
import importlib
import os
import sys
import types

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))  # the pin modules, whatever the import mode

import test_oracle_green as green  # noqa: E402
import test_oracle_hermitian as herm  # noqa: E402
import test_oracle_leads as leads_t  # noqa: E402
import test_oracle_nd_reference as ndr  # noqa: E402
import test_oracle_ribbon as ribbon  # noqa: E402
import test_oracle_scba as scba_t  # noqa: E402
import test_oracle_sp as sp_t  # noqa: E402

PINS = {
    "dense": [green.test_invariants_superlattice_dense, green.test_uniform_chain_closed_form,
              green.test_landauer_equals_transfer_matrix, green.test_meir_wingreen_equals_landauer_and_conservation,
              green.test_rgf_equals_dense_superlattice, green.test_density_uniform_chain_closed_form],
    "problem": [green.test_invariants_superlattice_dense, green.test_uniform_chain_closed_form,
                green.test_meir_wingreen_equals_landauer_and_conservation, green.test_rgf_equals_dense_superlattice,
                green.test_sampled_equals_dense, green.test_density_uniform_chain_closed_form,
                scba_t.test_fixed_point_conserves_current],
    "selfenergy": [leads_t.test_fermi_limits, green.test_invariants_superlattice_dense,
                   green.test_uniform_chain_closed_form, green.test_meir_wingreen_equals_landauer_and_conservation,
                   green.test_density_uniform_chain_closed_form, scba_t.test_fixed_point_conserves_current],
    "leads": [leads_t.test_modes_satisfy_dyson_fd_lead, leads_t.test_decimation_equals_modes_fd_lead,
              leads_t.test_decimation_satisfies_dyson_cnt_lead, leads_t.test_chain_lead_closed_form,
              green.test_uniform_chain_closed_form, green.test_uniform_wire_mode_sum],
    "observables": [green.test_landauer_equals_transfer_matrix, green.test_meir_wingreen_equals_landauer_and_conservation,
                    green.test_density_uniform_chain_closed_form, ribbon.test_perfect_ribbon_transmits_whole_channels],
    "rgf": [green.test_rgf_equals_dense_superlattice, green.test_rgf_equals_dense_cnt, ndr.test_layer_partition_is_rgf],
    "sampled": [green.test_sampled_equals_dense],
    "transfer": [green.test_landauer_equals_transfer_matrix],
    "nd_reference": [ndr.test_nd_reference_equals_dense, ndr.test_appendix_a_block_patterns,
                     ndr.test_layer_partition_is_rgf],
    "scba": [scba_t.test_fixed_point_conserves_current, scba_t.test_zero_strength_is_ballistic,
             scba_t.test_iteration_contracts],
    "response": [sp_t.test_jacobian_central_differences, sp_t.test_adjoint_and_forward_terms_against_jacobian],
    "poisson": [sp_t.test_poisson_eigenfunctions],
    "sp": [sp_t.test_newton_converges],
    "hermitian": [herm.test_zero_field_equals_the_symmetric_oracle, herm.test_gauge_covariance,
                  herm.test_reciprocity_under_field_reversal, herm.test_sum_rule_in_a_field,
                  herm.test_surface_green_fixed_point_with_complex_hopping, herm.test_quantum_hall_plateaus],
    "nd_general": [herm.test_general_nested_dissection_equals_the_definition,
                   herm.test_general_nested_dissection_reduces_to_the_symmetric_one],
}

# arguments of the parametrized pins (the first case of each parametrization
# unless a later one is the one that can see the mistake)
ARGS = {
    green.test_landauer_equals_transfer_matrix: [(0.25,), (-0.4,)],
    green.test_rgf_equals_dense_superlattice: [(5e-3,), (0.0,)],
    green.test_invariants_superlattice_dense: [(4e-3,), (0.0,)],
    leads_t.test_modes_satisfy_dyson_fd_lead: [(0.31,), (2.0,)],
    leads_t.test_decimation_equals_modes_fd_lead: [(0.3,)],
    leads_t.test_decimation_satisfies_dyson_cnt_lead: [(0.4,)],
    leads_t.test_chain_lead_closed_form: [(0.9,)],
    ribbon.test_perfect_ribbon_transmits_whole_channels: [(5,)],
    ndr.test_nd_reference_equals_dense: [(12, 10, 8, 3e-3)],
    scba_t.test_fixed_point_conserves_current: [(0.9,)],
    sp_t.test_poisson_eigenfunctions: [(9, 4, 3, 2)],
    herm.test_general_nested_dissection_equals_the_definition: [(16, 8, 12, 0.06)],
}

# (module, original text, planted mistake, what the mistake is)
MUTATIONS = [
    ("dense", 'Gl = G @ dense_sigma(dev, terms, "lesser") @ Ga', 'Gl = G @ dense_sigma(dev, terms, "lesser") @ G',
     "G^r in place of G^a"),
    ("dense", 'Gg = G @ dense_sigma(dev, terms, "greater") @ Ga', 'Gg = G @ dense_sigma(dev, terms, "lesser") @ Ga',
     "Sigma^< in place of Sigma^>"),
    ("problem", "A[np.ix_(idx, idx)] -= s", "A[np.ix_(idx, idx)] += s", "sign of the contact self-energy"),
    ("problem", "A[np.diag_indices(dev.n)] += terms.E + 1j * tr.eta", "A[np.diag_indices(dev.n)] += terms.E - 1j * tr.eta",
     "sign of eta"),
    ("problem", "A[np.diag_indices(dev.n)] -= terms.ph_r", "A[np.diag_indices(dev.n)] += terms.ph_r",
     "sign of the phonon self-energy"),
    ("problem", 'ph = terms.ph_lesser if which == "lesser" else terms.ph_greater',
     'ph = terms.ph_greater if which == "lesser" else terms.ph_lesser', "phonon Sigma^< and Sigma^> swapped"),
    ("problem", "f = [selfenergy.fermi(E, mu, tr.kT) for mu in tr.mu]",
     "f = [selfenergy.fermi(E, mu, tr.kT) for mu in tr.mu[::-1]]", "Fermi levels of the contacts swapped"),
    ("selfenergy", "return ex / (1.0 + ex)", "return 1.0 / (1.0 + ex)", "Fermi function branch"),
    ("selfenergy", "return 1j * f * broadening(sigma_r)", "return -1j * f * broadening(sigma_r)", "sign of Sigma^<"),
    ("selfenergy", "return -1j * (1.0 - f) * broadening(sigma_r)", "return -1j * f * broadening(sigma_r)",
     "occupation of Sigma^>"),
    ("selfenergy", "r = np.full(n, -0.5j * gamma_ph)", "r = np.full(n, -1j * gamma_ph)",
     "phonon Sigma^r without the 1/2"),
    ("leads", "lam = np.where(np.abs(lam1) < 1.0, lam1, lam2)", "lam = np.where(np.abs(lam1) > 1.0, lam1, lam2)",
     "growing root of the mode equation"),
    ("leads", "g_modes = lam / hop", "g_modes = lam * hop", "mode Green's function scale"),
    ("leads", "eps = eps + agb + bga", "eps = eps + agb", "dropped decimation term"),
    ("leads", "beta = H01.T.astype(complex).copy()", "beta = H01.astype(complex).copy()",
     "H01 in place of H10 = H01^T"),
    ("observables", "w[1:] += 0.5 * d", "pass", "dropped half of the trapezoid weights"),
    ("observables", "return 2.0 * (w[:, None] * Gl_diag.imag)", "return 1.0 * (w[:, None] * Gl_diag.imag)",
     "spin factor"),
    ("observables", "(w[:, None] * Gl_diag.imag)", "(w[:, None] * Gl_diag.real)", "real part for the imaginary one"),
    ("observables", "sigma_lesser_c @ Gg_cc - sigma_greater_c @ Gl_cc", "sigma_lesser_c @ Gg_cc + sigma_greater_c @ Gl_cc",
     "sign in the current"),
    ("observables", "gL @ G_LR @ gR @ G_LR.conj().T", "gL @ G_LR @ gR @ G_LR.T", "G^r in place of G^a"),
    ("rgf", "g[k] = np.linalg.inv(A[k] - tau[k - 1].T @ g[k - 1] @ tau[k - 1])",
     "g[k] = np.linalg.inv(A[k] + tau[k - 1].T @ g[k - 1] @ tau[k - 1])", "sign of the fold"),
    ("rgf", "Sk_l = Sl[k] + tau[k - 1].T @ gl[k - 1] @ tau[k - 1]", "Sk_l = Sl[k]", "dropped lesser fold term"),
    ("rgf", " + gl[k] @ t @ G.conj().T @ tT @ gka)", ")", "dropped lesser extraction term"),
    ("rgf", "X = gk @ t  # g_k tau_k", "X = gk @ tT  # g_k tau_k", "transposed coupling"),
    ("sampled", 'out["Gg"][s] = x @ (Sg @ x.conj())', 'out["Gg"][s] = x @ (Sl @ x.conj())', "Sigma^< for G^>"),
    ("sampled", "A.setdiag(A.diagonal() - terms.ph_r)", "A.setdiag(A.diagonal() + terms.ph_r)",
     "sign of the phonon self-energy"),
    ("transfer", "return float(1.0 / abs(A) ** 2)", "return float(1.0 / abs(A))", "amplitude for intensity"),
    ("transfer", "psi_prev = ((eps(j) - E) / t) * psi - psi_next", "psi_prev = ((E - eps(j)) / t) * psi - psi_next",
     "sign of the recurrence"),
    ("nd_reference", "Ab[j, k] = Ab[j, k] + self.Psi[i, j].T @ Ab[i, k]",
     "Ab[j, k] = Ab[j, k] - self.Psi[i, j].T @ Ab[i, k]", "sign of the Schur update"),
    ("nd_reference", "Gb[j, i] = Gb[i, j].T", "Gb[j, i] = Gb[i, j].conj().T", "G_ji as the adjoint"),
    ("nd_reference", "Pb[j, i] = -Pb[i, j].conj().T", "Pb[j, i] = Pb[i, j].conj().T", "sign of P_ji"),
    ("nd_reference", "S[np.ix_(C[i], C[i])] @ g.conj()", "S[np.ix_(C[i], C[i])] @ g", "G in place of G^a in N"),
    ("nd_reference", "acc = acc + self.Psi[i, j] @ Gb[j, i]", "acc = acc", "dropped diagonal extraction term"),
    ("scba", "new = [D * np.diag(G), D * np.diag(Gl), D * np.diag(Gg)]",
     "new = [D * np.diag(G), D * np.diag(Gg), D * np.diag(Gl)]", "lesser and greater swapped"),
    ("scba", "i_ph = np.sum(terms.ph_lesser * np.diag(Gg) - terms.ph_greater * np.diag(Gl))",
     "i_ph = np.sum(terms.ph_lesser * np.diag(Gg) + terms.ph_greater * np.diag(Gl))", "sign of the scattering current"),
    ("scba", "cur.append(np.trace(sl @ Gg[cc] - sg @ Gl[cc]))", "cur.append(np.trace(sl @ Gl[cc] - sg @ Gg[cc]))",
     "G^< and G^> swapped in the current"),
    ("response", "chi += w[e] * np.imag(G * Gl.T + Gl * G.conj())", "chi += w[e] * np.imag(G * Gl.T - Gl * G.conj())",
     "sign of the G^a term"),
    ("response", "vals[dev.rowptr[j] + hit[0]] += U[j]", "vals[dev.rowptr[j] + hit[0]] -= U[j]", "sign of U"),
    ("response", "Z = G @ (c[:, None] * Uc.conj())", "Z = G @ (c[:, None] * Uc)", "dropped conjugate (adjoint)"),
    ("response", 'np.einsum("ja,ab,jb->j", Wm, S, Uc.conj())', 'np.einsum("ja,ab,jb->j", Wm, S, Uc)',
     "dropped conjugate (forward)"),
    ("poisson", "                    continue  # Neumann", "                    diag += 1.0\n                    continue  # Neumann",
     "Dirichlet in place of Neumann"),
    ("poisson", "vals.append(-1.0)", "vals.append(1.0)", "sign of the coupling"),
    ("sp", "J = K - lam * response.jacobian(dev, tr, U)", "J = K + lam * response.jacobian(dev, tr, U)",
     "sign of the Jacobian's density term"),
    ("sp", "U = U - np.linalg.solve(J, F)", "U = U + np.linalg.solve(J, F)", "sign of the Newton step"),
    ("hermitian", "return lead.tau @ g @ lead.tau.conj().T", "return lead.tau @ g @ lead.tau.T",
     "tau^T in place of tau^dagger"),
    ("hermitian", "beta = H01.conj().T.astype(complex).copy()", "beta = H01.T.astype(complex).copy()",
     "H01^T in place of H01^dagger"),
    ("hermitian", "Ga = G.conj().T", "Ga = G.conj()", "conjugate in place of the adjoint"),
    ("hermitian", "@ selfenergy.broadening(sR) @ G_LR.conj().T", "@ selfenergy.broadening(sR) @ G_LR.T",
     "G^r in place of G^a in the transmission"),
    ("nd_general", "+ self.PsiL[j, i] @ Nb", "+ self.PsiR[i, j].T @ Nb", "right factor for the left one"),
    ("nd_general", "self.G0[j, i].conj().T for (i, j)", "self.G0[i, j].conj() for (i, j)", "N from G_ij"),
    ("nd_general", "Gb[i, j], Gb[j, i] = up[j], low[j]", "Gb[i, j], Gb[j, i] = up[j], up[j].T", "G_ji as G_ij^T"),
    ("nd_general", "Ab[j, k] = Ab[j, k] + Ab[j, i] @ self.PsiR[i, k]",
     "Ab[j, k] = Ab[j, k] + Ab[i, j].T @ self.PsiR[i, k]", "Schur update with A_ij^T"),
]


def _plant(monkeypatch, modname: str, old, new) -> None:
    """Compile the module with ``old`` replaced by ``new`` (unchanged for
    ``old=None``) and put its functions and classes in place of the originals
    in every oracle and pin module that holds them (including names bound by
    ``from .x import y``)."""
    mod = importlib.import_module("oracle." + modname)
    with open(mod.__file__) as fh:
        src = fh.read()
    if old is not None:
        assert src.count(old) == 1, (modname, old)
        src = src.replace(old, new)
    mut = types.ModuleType(mod.__name__)
    mut.__dict__.update(__file__=mod.__file__, __package__="oracle", __spec__=mod.__spec__)
    exec(compile(src, mod.__file__, "exec"), mut.__dict__)
    swap = {id(obj): mut.__dict__[name] for name, obj in vars(mod).items()
            if getattr(obj, "__module__", None) == mod.__name__ and name in mut.__dict__}
    for m in list(sys.modules.values()):
        name = getattr(m, "__name__", "") or ""
        if not (name == "oracle" or name.startswith("oracle.") or name.startswith("test_oracle_")):
            continue
        for attr, obj in list(vars(m).items()):
            if id(obj) in swap:
                monkeypatch.setattr(m, attr, swap[id(obj)])


def _run_pins(modname: str) -> list:
    """Run the pins of a module; returns the failures (pin name, exception)."""
    failed = []
    for pin in PINS[modname]:
        for args in ARGS.get(pin, [()]):
            try:
                with np.errstate(all="ignore"):
                    pin(*args)
            except Exception as exc:  # any failure counts: an assertion, a singular matrix, a shape error
                failed.append((pin.__name__, args, type(exc).__name__))
    return failed


@pytest.mark.parametrize("modname", sorted(PINS))
def test_control_without_a_mistake(monkeypatch, modname):
    """The harness itself (recompiling the module unchanged and swapping it in)
    fails no pin."""
    _plant(monkeypatch, modname, None, None)
    assert _run_pins(modname) == []


def test_every_module_has_mutations():
    assert {m for m, *_ in MUTATIONS} == set(PINS)


@pytest.mark.parametrize("modname,old,new,what", MUTATIONS, ids=[f"{m}:{w}" for m, _, _, w in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, modname, old, new, what):
    _plant(monkeypatch, modname, old, new)
    assert _run_pins(modname), f"no pin of oracle.{modname} catches: {what}"
