"""Input checks of the boundary, on the host (no GPU): nd_factor's H values and
contact blocks Sigma^r must be (complex) symmetric, because the fold is an
LDL^T elimination of A = A^T (paper Sec. 3.1); nd_diag_green's Sigma^< and
Sigma^> must be skew-Hermitian (Sec. 3.1, Eq. (5)-(6)).  The same routines run
inside nd_factor / nd_diag_green on host arrays, and as kernels on device
arrays (tests/test_gpu_checks.py).  One test per error code: a valid input
passes, and each kind of violation is rejected with its code."""
import numpy as np
import pytest

from oracle import problem
from paper_1305_1070_gb300 import build, ndgf, workloads

NOT_SYMMETRIC, NOT_SKEW = 2, 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _setup(n_e=3):
    dev = workloads.superlattice(12, 5, disorder=0.03, seed=7)
    tr = workloads.Transport(energies=np.linspace(0.05, 0.4, n_e))
    cp = np.concatenate([[0], np.cumsum([len(c) for c in dev.contacts])])
    plan = ndgf.nd_analyze(dev.n, dev.rowptr, dev.colind, cp, np.concatenate(dev.contacts), dev.coords, 16)
    terms = [problem.energy_terms(dev, tr, float(E)) for E in tr.energies]
    pack = lambda key: np.stack([np.concatenate([s.ravel() for s in getattr(t, key)]) for t in terms])
    return dev, plan, pack("sigma_r"), pack("sigma_lesser"), pack("sigma_greater")


def _status(fn, *args):
    try:
        fn(*args)
        return 0
    except ndgf.NDError as e:
        return e.status


def test_valid_inputs_pass():
    dev, plan, sr, sl, sg = _setup()
    n_e = sr.shape[0]
    assert _status(ndgf.nd_check_factor_inputs, plan, dev.values, sr, n_e) == 0
    ph_l = np.full((n_e, dev.n), 0.01j)
    assert _status(ndgf.nd_check_lesser_inputs, plan, sl, sg, ph_l, -ph_l, n_e) == 0
    assert _status(ndgf.nd_check_lesser_inputs, plan, None, None, None, None, n_e) == 0


def test_not_symmetric():
    dev, plan, sr, _, _ = _setup()
    n_e = sr.shape[0]
    # an off-diagonal H value that differs from its transposed entry
    H = dev.values.copy()
    r = 3
    q = next(q for q in range(dev.rowptr[r], dev.rowptr[r + 1]) if dev.colind[q] != r)
    H[q] *= 1.0 + 1e-6
    assert _status(ndgf.nd_check_factor_inputs, plan, H, sr, n_e) == NOT_SYMMETRIC
    # a non-finite H value
    H = dev.values.copy()
    H[q] = np.nan
    assert _status(ndgf.nd_check_factor_inputs, plan, H, sr, n_e) == NOT_SYMMETRIC
    # a contact block that is Hermitian-like instead of complex symmetric (one entry pair changed)
    m = len(dev.contacts[1])
    m0 = len(dev.contacts[0])
    bad = sr.copy()
    bad[2, 0 * m0 + 1] = np.conj(bad[2, 1 * m0 + 0]) + 1e-3  # first contact block, entry (0, 1)
    assert _status(ndgf.nd_check_factor_inputs, plan, dev.values, bad, n_e) == NOT_SYMMETRIC
    # a change at the rounding level passes (relative tolerance 1e-8 of the block's largest entry)
    ok = sr.copy()
    ok[1, m0 * m0 + 1] *= 1.0 + 1e-13
    assert m == m0 and _status(ndgf.nd_check_factor_inputs, plan, dev.values, ok, n_e) == 0


def test_not_skew_hermitian():
    dev, plan, sr, sl, sg = _setup()
    n_e = sr.shape[0]
    gamma = 1j * (sr - 0.0)  # not skew-Hermitian in general: i Sigma^r is neither
    assert _status(ndgf.nd_check_lesser_inputs, plan, gamma, sg, None, None, n_e) == NOT_SKEW
    # Gamma itself (Hermitian) passed as Sigma^> instead of -i (1 - f) Gamma
    m0 = len(dev.contacts[0])
    herm = sg / (-1j)
    assert _status(ndgf.nd_check_lesser_inputs, plan, sl, herm, None, None, n_e) == NOT_SKEW
    # one entry pair broken
    bad = sl.copy()
    bad[0, 1] += 1e-3 * np.abs(sl[0, :m0 * m0]).max()
    assert _status(ndgf.nd_check_lesser_inputs, plan, bad, sg, None, None, n_e) == NOT_SKEW
    # a phonon diagonal with a real part
    ph = np.full((n_e, dev.n), 0.01j)
    ph[1, 5] += 1e-4
    assert _status(ndgf.nd_check_lesser_inputs, plan, sl, sg, ph, -ph.conj(), n_e) == NOT_SKEW
    ph = np.full((n_e, dev.n), 0.01j)
    ph[2, 0] = np.nan
    assert _status(ndgf.nd_check_lesser_inputs, plan, None, None, None, ph, n_e) == NOT_SKEW


def test_bad_arguments():
    dev, plan, sr, _, _ = _setup()
    assert _status(ndgf.nd_check_factor_inputs, plan, None, sr, 3) == 1
    assert _status(ndgf.nd_check_factor_inputs, plan, dev.values, None, 3) == 1  # contacts need Sigma^r
    assert _status(ndgf.nd_check_lesser_inputs, plan, None, None, None, None, -1) == 1


def test_complex_hamiltonian_is_rejected_not_cast():
    """A device in a magnetic field (Peierls phases: complex hoppings, a
    Hermitian H that is not complex symmetric) is rejected with
    ND_ERR_NOT_SYMMETRIC by the binding, the lead constructor and the Solver,
    before anything reaches the library or the GPU: a cast to float64 would
    drop the phases and solve another problem.  The same device without a
    field but stored as complex is rejected too; its real part passes."""
    from paper_1305_1070_gb300.solver import Solver
    dev = workloads.magnetic_superlattice(12, 5, 0.05, disorder=0.03, seed=7)
    tr = workloads.Transport(energies=np.array([0.3]))
    assert np.iscomplexobj(dev.values) and np.abs(dev.values.imag).max() > 0.1
    cp = np.concatenate([[0], np.cumsum([len(c) for c in dev.contacts])])
    plan = ndgf.nd_analyze(dev.n, dev.rowptr, dev.colind, cp, np.concatenate(dev.contacts), dev.coords, 16)
    sr = np.zeros((1, sum(len(c) ** 2 for c in dev.contacts)), dtype=complex)
    assert _status(ndgf.nd_check_factor_inputs, plan, dev.values, sr, 1) == NOT_SYMMETRIC
    lead = dev.leads[0]
    assert np.iscomplexobj(lead.H01)
    assert _status(ndgf.nd_lead_create, lead.H00, lead.H01, lead.tau) == NOT_SYMMETRIC
    assert _status(Solver, dev, tr) == NOT_SYMMETRIC
    zero = workloads.magnetic_superlattice(12, 5, 0.0, disorder=0.03, seed=7)
    assert _status(ndgf.nd_check_factor_inputs, plan, zero.values, sr, 1) == NOT_SYMMETRIC
    _, _, sr_real, _, _ = _setup(1)
    assert _status(ndgf.nd_check_factor_inputs, plan, zero.values.real, sr_real, 1) == 0
    with pytest.raises(ndgf.NDError) as err:
        ndgf.require_real(np.zeros(4, dtype=np.float32).view(np.complex64), "x")
    assert err.value.status == NOT_SYMMETRIC
    assert ndgf.require_real(np.arange(3), "x").dtype == np.float64


def test_binding_checks_buffers_before_the_library():
    """The C ABI takes raw pointers and cannot see buffer sizes or element
    types; the binding checks them against the plan (nnz, n, contact blocks)
    and the handle's energies, so that a short buffer is refused instead of
    overrun and a narrower type is refused instead of misread.  A handle
    without a workspace (NULL) shows which side answered: the binding's
    messages name the buffer, the library's names the NULL handle."""
    dev, plan, sr, sl, sg = _setup(n_e=3)
    fact = ndgf.Fact(None, plan)
    fact.max_ne, fact.n_e = 3, 3
    E = np.linspace(0.05, 0.4, 3)
    n = dev.n

    def msg(fn, *args):
        with pytest.raises(ndgf.NDError) as err:
            fn(*args)
        assert err.value.status == 1
        return str(err.value)

    assert "NULL" in msg(ndgf.nd_factor, fact, dev.values, sr, None, E, 3, 1e-6)
    assert "sigma_r" in msg(ndgf.nd_factor, fact, dev.values, sr[:2], None, E, 3, 1e-6)
    assert "H_values" in msg(ndgf.nd_factor, fact, dev.values[:-1], sr, None, E, 3, 1e-6)
    assert "energies" in msg(ndgf.nd_factor, fact, dev.values, sr, None, E.astype(np.float32), 3, 1e-6)
    assert "sigma_ph_r" in msg(ndgf.nd_factor, fact, dev.values, sr, np.zeros((3, n), np.complex64), E, 3, 1e-6)
    fact.n_e = 3
    out = [np.zeros((3, n), dtype=np.complex128) for _ in range(3)]
    assert "NULL" in msg(ndgf.nd_diag_green, fact, sl, sg, None, None, *out)
    assert "Gl" in msg(ndgf.nd_diag_green, fact, sl, sg, None, None, out[0], out[1][:2], out[2])
    wide = np.zeros((3, 2 * n), dtype=np.complex128)
    assert "Gg" in msg(ndgf.nd_diag_green, fact, sl, sg, None, None, out[0], out[1], wide[:, ::2])
    assert "sigma_greater" in msg(ndgf.nd_diag_green, fact, sl, sg.astype(np.complex64), None, None, *out)
    assert "cert" in msg(ndgf.nd_certificate, fact, np.zeros((2, 8)))
    assert "weights" in msg(ndgf.nd_fact_density, fact, np.ones(2), 1.0, 0, np.zeros(n))
    assert "out" in msg(ndgf.nd_fact_density, fact, np.ones(3), 1.0, 0, np.zeros(n, dtype=np.float32))
    # float64 views of complex buffers are the ABI's own layout and pass
    assert "NULL" in msg(ndgf.nd_diag_green, fact, sl.view(np.float64), sg, None, None, *out)


def test_binding_checks_the_epilogue_buffers():
    """The same buffer checks on the density, current and response entry
    points: short or narrower arrays are refused by the binding (their
    messages name the buffer); well-formed ones reach the library, which here
    refuses the NULL handle or the host arrays that these calls do not take."""
    dev, plan, _, _, _ = _setup(n_e=3)
    fact = ndgf.Fact(None, plan)
    fact.max_ne, fact.n_e = 3, 3
    n = dev.n

    def msg(fn, *args):
        with pytest.raises(ndgf.NDError) as err:
            fn(*args)
        assert err.value.status == 1
        return str(err.value)

    Gl = np.zeros((3, n), dtype=np.complex128)
    assert "density: Gl: " in msg(ndgf.nd_density, Gl[:2], np.ones(3), 3, n, 1.0, 0, np.zeros(n))
    assert "density: weights: " in msg(ndgf.nd_density, Gl, np.ones(3, dtype=np.float32), 3, n, 1.0, 0, np.zeros(n))
    assert "density: out: " in msg(ndgf.nd_density, Gl, np.ones(3), 3, n, 1.0, 0, np.zeros(n - 1))
    assert "current: 16 bytes" in msg(ndgf.nd_contact_current, fact, 0, np.zeros(2))
    assert "current_im: elements of type complex128" in msg(ndgf.nd_contact_current, fact, 0, np.zeros(3), np.zeros(3, dtype=np.complex128))
    assert "t_out: " in msg(ndgf.nd_density_gradient, fact, np.ones(n), np.zeros((2, n), dtype=np.complex128))
    assert "gradient: c: " in msg(ndgf.nd_density_gradient, fact, np.ones(n - 1), np.zeros((3, n), dtype=np.complex128))
    assert "jvp: v: elements" in msg(ndgf.nd_density_jvp, fact, np.ones(n, dtype=np.complex128), np.zeros((3, n), dtype=np.complex128))
    for fn, args in ((ndgf.nd_contact_current, (fact, 0, np.zeros(3))),
                     (ndgf.nd_density_gradient, (fact, np.ones(n), np.zeros((3, n), dtype=np.complex128))),
                     (ndgf.nd_density_jvp, (fact, np.ones(n), np.zeros((3, n), dtype=np.complex128)))):
        assert "bytes" not in msg(fn, *args) and "type" not in msg(fn, *args)


class _NoDevice:
    """The real library for the host-only calls (analysis, plan queries,
    errors); every call that needs a device returns ND_OK without doing
    anything.  It lets the driver's call sequences run on the CPU to show
    that the buffers it allocates pass the binding's checks."""
    DEVICE = {"nd_fact_create", "nd_fact_destroy", "nd_factor", "nd_diag_green", "nd_certificate",
              "nd_contact_current", "nd_autotune", "nd_density_gradient", "nd_density_jvp", "nd_fact_density",
              "nd_density", "nd_lead_create", "nd_lead_destroy", "nd_lead_sigma", "nd_sigma_lesser_fermi",
              "nd_phonon_const", "nd_phonon_scba"}

    def __init__(self, real):
        self.real = real

    def __getattr__(self, name):
        if name in self.DEVICE:
            return lambda *args: 0
        return getattr(self.real, name)


@pytest.mark.parametrize("case", ["superlattice", "phonons", "cnt", "union"])
def test_driver_buffers_pass_the_binding_checks(monkeypatch, case):
    """The Solver's own buffers (device ones here allocated on the CPU) and
    its call sequences -- step, the host-buffer step, certificate, contact
    currents, tuner, adjoint and forward products, densities -- pass every
    check of the binding, at a full batch and at a shorter last chunk."""
    from paper_1305_1070_gb300.solver import Solver
    import torch
    monkeypatch.setattr(ndgf, "_LIB", _NoDevice(ndgf.lib()))
    if case == "cnt":
        dev = workloads.cnt_zigzag(3, disorder=0.05, seed=1)
        tr = workloads.Transport(energies=np.linspace(-0.5, 0.5, 5))
    elif case == "union":
        dev = workloads.union([workloads.superlattice(12, 4, disorder=0.02, seed=s) for s in (1, 2, 3)])
        tr = workloads.Transport(energies=np.linspace(0.05, 0.4, 5))
    else:
        dev = workloads.superlattice(16, 6, disorder=0.03, seed=3)
        tr = workloads.Transport(energies=np.linspace(0.05, 0.4, 5), gamma_ph=3e-3 if case == "phonons" else 0.0)
    s = Solver(dev, tr, leaf_size=8, max_ne=4, delay=2, adjoint=case not in ("phonons", "union"), device="cpu")
    if case == "superlattice":
        s.set_potential(np.full(dev.n, 0.01))
    for E in (tr.energies[:4], tr.energies[4:]):
        k = len(E)
        s.step(E)
        assert s.fact.n_e == k
        s.certificate(k)
        s.current(0, k), s.current(1, k)
        out = [torch.zeros(k, dev.n, dtype=torch.complex128) for _ in range(3)]
        s.step_host(torch.as_tensor(E), *out, H_host=torch.as_tensor(dev.values))
        w = torch.full((k,), 0.01, dtype=torch.float64)
        dens = torch.zeros(dev.n, dtype=torch.float64)
        ndgf.nd_fact_density(s.fact, w, 1.0, 0, dens)
        ndgf.nd_density(s.Gl[:k], w, k, dev.n, 1.0, 1, dens)
        if case not in ("phonons", "union"):
            s.density_gradient_terms(np.ones(dev.n), k)
            ndgf.nd_density_jvp(s.fact, torch.ones(dev.n, dtype=torch.float64),
                                torch.zeros(k, dev.n, dtype=torch.complex128))
    s.autotune(torch.as_tensor(tr.energies[:4]))
    assert s.fact.n_e == 4
    if case == "phonons":
        s.scba(tr.energies[:4], 0.01, updates=2)


def test_analysis_indices_fit_the_abi():
    """The graph's indices are int32 in the C ABI: values that do not fit, or
    a non-integer array, are refused instead of wrapping in the cast."""
    dev = workloads.superlattice(6, 4)
    cp = np.array([0, 4, 8])
    ci = np.concatenate(dev.contacts)
    big = dev.rowptr.astype(np.int64).copy()
    big[-1] = 2 ** 31
    for args in ((big, dev.colind, cp, ci), (dev.rowptr, dev.colind.astype(np.float64), cp, ci),
                 (dev.rowptr, dev.colind, cp, ci - 1)):
        with pytest.raises(ndgf.NDError) as err:
            ndgf.nd_analyze(dev.n, *args, dev.coords, 8)
        assert err.value.status == 1
    assert ndgf.nd_plan_query(ndgf.nd_analyze(dev.n, dev.rowptr, dev.colind, cp, ci, dev.coords, 8))["n"] == dev.n


def test_energies_per_handle_fit_the_grid():
    """Energies index the y dimension of every launch grid (at most 65535):
    a larger workspace is refused before any allocation."""
    _, plan, _, _, _ = _setup(n_e=1)
    with pytest.raises(ndgf.NDError) as err:
        ndgf.nd_fact_create(plan, 65536, ndgf.ND_PREC_FP64)
    assert err.value.status == 8


def test_selected_entries_buffers():
    """nd_selected_entries: int32 pair lists of `count` entries, an int32
    counter and [n_e][count] complex outputs, checked by the binding."""
    _, plan, _, _, _ = _setup(n_e=3)
    fact = ndgf.Fact(None, plan)
    fact.max_ne, fact.n_e = 3, 3
    x = np.arange(5, dtype=np.int32)
    out = np.zeros((3, 5), dtype=np.complex128)
    miss = np.zeros(1, dtype=np.int32)

    def msg(*args):
        with pytest.raises(ndgf.NDError) as err:
            ndgf.nd_selected_entries(fact, *args)
        assert err.value.status == 1
        return str(err.value)

    assert "bad argument" in msg(x, x, 5, out, None, None, miss)  # the library: NULL handle
    assert "x: elements of type int64" in msg(x.astype(np.int64), x, 5, out, None, None, miss)
    assert "y: 4 elements" in msg(x, x[:4], 5, out, None, None, miss)
    assert "Gr: " in msg(x, x, 5, out[:2], None, None, miss)
    assert "n_missing" in msg(x, x, 5, out, None, None, np.zeros(1, dtype=np.int64))


def test_self_energy_builder_buffers():
    """The self-energy builders and the Born update: outputs hold [n_e] blocks
    of the contact sizes (or [n_e][n] diagonals) and the energies are float64,
    checked by the binding before the library sees the pointers."""
    n, n_e = 6, 3
    E = np.linspace(0.1, 0.3, n_e)
    sr = np.zeros((n_e, 2 * 9), dtype=np.complex128)

    def msg(fn, *args):
        with pytest.raises(ndgf.NDError) as err:
            fn(*args)
        assert err.value.status == 1
        return str(err.value)

    assert "sigma_lesser: " in msg(ndgf.nd_sigma_lesser_fermi, sr, n_e, [3, 3], [0.1, 0.0], 0.03, E, sr[:2], sr)
    assert "energies: elements of type complex128" in msg(ndgf.nd_sigma_lesser_fermi, sr, n_e, [3, 3], [0.1, 0.0],
                                                          0.03, E.astype(complex), sr, sr)
    ph = np.zeros((n_e, n), dtype=np.complex128)
    assert "ph_greater: " in msg(ndgf.nd_phonon_const, n, n_e, 0.01, 0.0, 0.03, E, ph, ph, ph[:, :3].copy())
    assert "stats: " in msg(ndgf.nd_phonon_scba, n, n_e, 0.01, 1.0, ph, ph, ph, ph, ph, ph, np.zeros(1))
    assert "Gl: " in msg(ndgf.nd_phonon_scba, n, n_e, 0.01, 1.0, ph, ph[:1], ph, ph, ph, ph, np.zeros(2))
    lead = ndgf.Lead(None)
    lead.m_c = 3
    out = np.zeros((n_e, 18), dtype=np.complex128)
    assert "sigma_out: " in msg(ndgf.nd_lead_sigma, lead, E, n_e, 1e-6, out, 18, 10)


def test_host_arrays_match_their_lengths():
    """Host arrays that the library reads by implied lengths (the graph, the
    contact lists, the coordinates, one Fermi level per contact) are checked
    against those lengths by the binding."""
    dev = workloads.superlattice(6, 4)
    cp = np.array([0, 4, 8])
    ci = np.concatenate(dev.contacts)
    bad = ((dev.n + 1, dev.rowptr, dev.colind, cp, ci, dev.coords),
           (dev.n, dev.rowptr, dev.colind[:-1], cp, ci, dev.coords),
           (dev.n, dev.rowptr, dev.colind, cp, ci[:7], dev.coords),
           (dev.n, dev.rowptr, dev.colind, cp, ci, dev.coords[:-1]))
    for args in bad:
        with pytest.raises(ndgf.NDError) as err:
            ndgf.nd_analyze(*args, 8)
        assert err.value.status == 1
    sr = np.zeros((1, 32), dtype=np.complex128)
    with pytest.raises(ndgf.NDError) as err:
        ndgf.nd_sigma_lesser_fermi(sr, 1, [4, 4], [0.1], 0.03, np.zeros(1), sr, sr)
    assert err.value.status == 1


def test_poisson_and_vector_buffers():
    """The Poisson operator and the vector operations: [batch][nx * ny] and
    [n] float64 buffers, checked by the binding (a handle without a workspace
    and the library's own refusal of host arrays show the rest reaches it)."""
    p = ndgf.Poisson(None)
    p.sites = 12

    def msg(fn, *args):
        with pytest.raises(ndgf.NDError) as err:
            fn(*args)
        assert err.value.status == 1
        return str(err.value)

    assert "u: 88 bytes" in msg(ndgf.nd_poisson_apply, p, np.zeros(11), np.zeros(12))
    assert "u: " in msg(ndgf.nd_poisson_solve, p, np.zeros(24), np.zeros(23), 2)
    assert "out: elements of type float32" in msg(ndgf.nd_vec_dot, np.zeros(4), np.zeros(4), 4,
                                                  np.zeros(1, dtype=np.float32))
    assert "y: 24 bytes" in msg(ndgf.nd_vec_axpby, 1.0, np.zeros(4), 1.0, np.zeros(3), 4)
    assert "d: " in msg(ndgf.nd_vec_mul, np.zeros(3), np.zeros(4), np.zeros(4), 4)
    assert "x: elements of type complex128" in msg(ndgf.nd_vec_scale_pos, 1.0, np.zeros(4, complex), np.zeros(4), 4)
    # well-formed host arrays reach the library, which takes device arrays only
    assert "bytes" not in msg(ndgf.nd_vec_axpby, 1.0, np.zeros(4), 1.0, np.zeros(4), 4)


def test_noalloc_buffers():
    """The allocation-free inversion: A holds batch x n x n complex64 in one
    block and the singular counter is int32, checked by the binding; sizes
    beyond the library's cap are left to the library's own refusal."""
    def msg(*args):
        with pytest.raises(ndgf.NDError) as err:
            ndgf.nd_invert_c64_noalloc(*args)
        assert err.value.status == 1
        return str(err.value)

    cnt = np.zeros(1, dtype=np.int32)
    assert "complex64" in msg(np.zeros((1, 8, 8), dtype=np.complex128), 8, 1, cnt)
    assert "contiguous" in msg(np.zeros((1, 8, 7), dtype=np.complex64), 8, 1, cnt)
    assert "n_singular" in msg(np.zeros((1, 8, 8), dtype=np.complex64), 8, 1, np.zeros(1, dtype=np.int64))
    assert "must be device arrays" in msg(np.zeros((1, 8, 8), dtype=np.complex64), 8, 1, cnt)  # well formed: the library
    assert "complex64" not in msg(np.zeros(1, dtype=np.complex64), 513, 1, cnt)  # over the cap: the library
