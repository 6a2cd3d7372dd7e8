"""Seeded synthetic device workloads (inputs only, no Green's-function arithmetic).

This module builds the *inputs* of the nested-dissection NEGF path: the sparse
real-symmetric Hamiltonian H of a device, the site coordinates, the contact site
sets, the description of the semi-infinite leads and the transport parameters.
It is shared by the CUDA path and by the CPU oracle, so it holds none of the
method's arithmetic: no self-energy, no Fermi function, no Green's function.

Devices (paper Sec. 2, Fig. 1-2 and Sec. 4.2):

* ``superlattice`` -- 2D five-point finite-difference effective-mass device
  (Sec. 4.2.1): transport length ``L`` columns, transverse width ``W`` rows,
  hard-wall transverse boundaries, a barrier/well potential along transport and
  optional uniform on-site disorder.  Leads are flat (V = 0) semi-infinite
  copies of one column attached at column 0 and column L-1.
* ``cnt_zigzag`` -- (n,0) carbon nanotube with one p_z orbital per atom and
  nearest-neighbour hopping (tight binding, Sec. 4.2.2 uses the same model on a
  planar ribbon).  Rings of n atoms are the transport layers; the leads are
  perfect semi-infinite tubes.
* ``agnr`` -- planar armchair graphene nanoribbon, one p_z orbital per atom,
  nearest-neighbour hopping -3.1 eV, on-site 0 (Sec. 4.2.2); atom columns are
  the transport layers, four per cell, and the leads are perfect ribbons.
* ``chain`` -- 1D tight-binding chain (W = 1), used for closed-form checks.

Site order ("caller order"): transport layer by layer, so that layer ``k``
occupies a contiguous index range.  All arrays are numpy; CSR column indices
are sorted and the diagonal is always stored.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# hbar^2 / (2 m_e) in eV nm^2 (CODATA 2018: hbar^2/(2 m_e) = 3.80998212e-20 eV m^2).
HBAR2_2ME_EV_NM2 = 0.0380998212
# Boltzmann constant in eV/K.
KB_EV = 8.617333262e-5


@dataclasses.dataclass
class Lead:
    """A semi-infinite periodic lead.

    ``H00`` is the on-site block of one principal layer (m x m, real symmetric),
    ``H01`` the hopping from a principal layer to the next one *away* from the
    device (m x m), and ``tau`` the coupling from the contact sites of the device
    (rows, in the order of the device contact set) to the lead layer adjacent to
    the device (columns).  The retarded self-energy that the lead folds onto the
    contact sites is tau g_s tau^T, g_s the surface Green's function of the lead
    (paper Sec. 2: each semi-infinite lead enters only through a self-energy on
    the first or last device layer).
    """

    H00: np.ndarray
    H01: np.ndarray
    tau: np.ndarray
    hop: float | None = None  # set when H01 = -hop * I and tau = -hop * I


@dataclasses.dataclass
class Device:
    """Sparse device Hamiltonian plus everything the transport path needs."""

    name: str
    n: int
    rowptr: np.ndarray  # int32 [n+1]
    colind: np.ndarray  # int32 [nnz]
    values: np.ndarray  # float64 [nnz], H in eV (complex128 for a Hermitian H with complex hoppings)
    coords: np.ndarray  # float64 [n, d], nm
    layers: list  # list of int arrays, transport layers in order
    contacts: list  # list of int arrays: contact site sets (left, right)
    leads: list  # list of Lead, one per contact
    transport_axis: int = 0

    @property
    def nnz(self) -> int:
        return int(self.colind.shape[0])

    def dense(self) -> np.ndarray:
        """Dense copy of H (only for small devices)."""
        Hd = np.zeros((self.n, self.n), dtype=self.values.dtype)
        for r in range(self.n):
            s, e = self.rowptr[r], self.rowptr[r + 1]
            Hd[r, self.colind[s:e]] = self.values[s:e]
        return Hd


def _csr_from_dict(n: int, entries: dict) -> tuple:
    rows = [[] for _ in range(n)]
    for (r, c), v in entries.items():
        rows[r].append((c, v))
    rowptr = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for r in range(n):
        rows[r].sort()
        for c, v in rows[r]:
            cols.append(c)
            vals.append(v)
        rowptr[r + 1] = len(cols)
    return rowptr, np.asarray(cols, dtype=np.int32), np.asarray(vals, dtype=np.float64)


def _csr_from_coo(n: int, r: np.ndarray, c: np.ndarray, v: np.ndarray) -> tuple:
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    return rowptr, c.astype(np.int32), v.astype(np.float64)


def fd_hopping(a_nm: float, m_eff: float) -> float:
    """Five-point stencil hopping t = hbar^2 / (2 m* a^2) in eV."""
    return HBAR2_2ME_EV_NM2 / (m_eff * a_nm * a_nm)


def superlattice_potential(L: int, a_nm: float, v_barrier: float, half_period_nm: float) -> np.ndarray:
    """Barrier/well profile along transport: column x is barrier when
    floor(x * a / half_period) is odd (a well first, starting at column 0)."""
    x = np.arange(L)
    return np.where((np.floor(x * a_nm / half_period_nm + 1e-9).astype(np.int64) % 2) == 1, v_barrier, 0.0)


def superlattice(L: int, W: int, *, a_nm: float = 0.5, m_eff: float = 0.067, v_barrier: float = 0.3,
                 half_period_nm: float = 2.0, disorder: float = 0.0, seed: int | None = None,
                 potential: np.ndarray | None = None) -> Device:
    """2D effective-mass superlattice on an L (transport) x W (transverse) grid.

    Site (x, y) has caller index x*W + y.  On-site 4t + V(x) + U(-disorder,
    +disorder); hopping -t to the four neighbours inside the device; hard-wall
    transverse edges.  Disorder draws come from numpy's PCG64 with ``seed``.
    ``potential`` (length L*W) overrides the profile when given.
    """
    t = fd_hopping(a_nm, m_eff)
    n = L * W
    if potential is None:
        V = np.repeat(superlattice_potential(L, a_nm, v_barrier, half_period_nm), W)
    else:
        V = np.asarray(potential, dtype=np.float64).reshape(n)
    if disorder > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        V = V + rng.uniform(-disorder, disorder, size=n)
    idx = np.arange(n).reshape(L, W)
    rs, cs, vs = [np.arange(n)], [np.arange(n)], [4.0 * t + V]
    # transport neighbours
    a, b = idx[:-1, :].ravel(), idx[1:, :].ravel()
    rs += [a, b]; cs += [b, a]; vs += [np.full(a.size, -t)] * 2
    # transverse neighbours
    a, b = idx[:, :-1].ravel(), idx[:, 1:].ravel()
    rs += [a, b]; cs += [b, a]; vs += [np.full(a.size, -t)] * 2
    rowptr, colind, values = _csr_from_coo(n, np.concatenate(rs), np.concatenate(cs), np.concatenate(vs))
    xs, ys = np.meshgrid(np.arange(L), np.arange(W), indexing="ij")
    coords = np.stack([xs.ravel() * a_nm, ys.ravel() * a_nm], axis=1).astype(np.float64)
    layers = [idx[x].copy() for x in range(L)]
    H00 = 4.0 * t * np.eye(W) - t * (np.eye(W, k=1) + np.eye(W, k=-1))
    lead = Lead(H00=H00, H01=-t * np.eye(W), tau=-t * np.eye(W), hop=t)
    lead_r = Lead(H00=H00.copy(), H01=-t * np.eye(W), tau=-t * np.eye(W), hop=t)
    return Device(name=f"superlattice_{L}x{W}", n=n, rowptr=rowptr, colind=colind, values=values,
                  coords=coords, layers=layers, contacts=[idx[0].copy(), idx[L - 1].copy()],
                  leads=[lead, lead_r])


def magnetic_superlattice(L: int, W: int, flux: float, **kw) -> Device:
    """The superlattice of ``superlattice`` (same keywords) in a uniform
    magnetic field perpendicular to the grid: a general Hermitian H, not
    complex symmetric (Peierls substitution in the Landau gauge A = (-B y, 0)).
    Every hopping along the transport direction from column x to x + 1 at row
    y gets the phase exp(i 2 pi flux y), flux = B a^2 / (h / e) the flux
    quantum fraction per plaquette; transverse hoppings keep no phase.  The
    gauge is uniform along transport, so the leads keep it: a lead's H01 and
    tau become -t diag(exp(+-i 2 pi flux y)), the sign set by the direction
    from the device outwards.  H values are complex128; the leads have no
    closed form (hop = None)."""
    dev = superlattice(L, W, **kw)
    t = fd_hopping(kw.get("a_nm", 0.5), kw.get("m_eff", 0.067))
    rows = np.repeat(np.arange(dev.n), np.diff(dev.rowptr))
    cols = dev.colind.astype(np.int64)
    ph = 2.0 * np.pi * flux
    values = dev.values.astype(np.complex128)
    fwd = cols + W == rows   # hopping from column x (col) to column x + 1 (row)
    bwd = rows + W == cols
    y = rows % W
    values[fwd] *= np.exp(1j * ph * y[fwd])
    values[bwd] *= np.exp(-1j * ph * y[bwd])
    D = np.exp(1j * ph * np.arange(W))
    H00 = dev.leads[0].H00
    left = Lead(H00=H00.copy(), H01=-t * np.diag(D), tau=-t * np.diag(D), hop=None)
    right = Lead(H00=H00.copy(), H01=-t * np.diag(D.conj()), tau=-t * np.diag(D.conj()), hop=None)
    return dataclasses.replace(dev, name=f"magnetic_superlattice_{L}x{W}", values=values, leads=[left, right])


def chain(N: int, *, t: float = 1.0, eps0: float = 0.0, potential: np.ndarray | None = None) -> Device:
    """1D chain: on-site eps0 + potential[j], hopping -t, leads = uniform chain."""
    V = np.zeros(N) if potential is None else np.asarray(potential, dtype=np.float64)
    ent = {}
    for j in range(N):
        ent[(j, j)] = eps0 + V[j]
        if j + 1 < N:
            ent[(j, j + 1)] = -t
            ent[(j + 1, j)] = -t
    rowptr, colind, values = _csr_from_dict(N, ent)
    coords = np.arange(N, dtype=np.float64).reshape(N, 1)
    lead = lambda: Lead(H00=np.array([[eps0]]), H01=np.array([[-t]]), tau=np.array([[-t]]), hop=t)
    return Device(name=f"chain_{N}", n=N, rowptr=rowptr, colind=colind, values=values, coords=coords,
                  layers=[np.array([j]) for j in range(N)], contacts=[np.array([0]), np.array([N - 1])],
                  leads=[lead(), lead()])


def _cnt_cell_coords(nring: int, acc: float) -> tuple:
    """Atoms of one (nring,0) unit cell: 4 rings, cell length 3*acc.

    Returns (z offsets per ring, angle offsets per ring in units of 2*pi/nring).
    Rings A, B, C, D at z = 0, acc/2, 3acc/2, 2acc; B and C are rotated by half
    an angular step.  A-B and C-D are zigzag bonds, B-C and D-A(next) axial.
    """
    return np.array([0.0, 0.5 * acc, 1.5 * acc, 2.0 * acc]), np.array([0.0, 0.5, 0.5, 0.0])


def cnt_zigzag(n_cells: int, *, nring: int = 10, t: float = -2.7, acc: float = 0.142,
               disorder: float = 0.0, seed: int | None = None) -> Device:
    """(nring,0) zigzag nanotube, n_cells cells of 4 rings (4*nring atoms each).

    Connectivity: pairs closer than 1.1*acc in 3D.  On-site 0 + U(-disorder,
    +disorder), hopping t (t = -2.7 eV gives H_ij = -2.7).  Caller order is
    ring by ring along the tube axis (z).
    """
    a = math.sqrt(3.0) * acc
    R = nring * a / (2.0 * math.pi)
    zoff, phoff = _cnt_cell_coords(nring, acc)
    nr = 4 * n_cells
    n = nr * nring
    coords = np.zeros((n, 3))
    for c in range(n_cells):
        for r in range(4):
            ring = 4 * c + r
            phi = (np.arange(nring) + phoff[r]) * 2.0 * math.pi / nring
            sl = slice(ring * nring, (ring + 1) * nring)
            coords[sl, 0] = R * np.cos(phi)
            coords[sl, 1] = R * np.sin(phi)
            coords[sl, 2] = c * 3.0 * acc + zoff[r]
    onsite = np.zeros(n)
    if disorder > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        onsite = onsite + rng.uniform(-disorder, disorder, size=n)
    rs, cs, vs = [np.arange(n)], [np.arange(n)], [onsite]
    cut = 1.1 * acc
    # neighbours only between adjacent rings (and within a ring, none exist)
    for ring in range(nr - 1):
        A = np.arange(ring * nring, (ring + 1) * nring)
        B = np.arange((ring + 1) * nring, (ring + 2) * nring)
        d = np.linalg.norm(coords[A][:, None, :] - coords[B][None, :, :], axis=2)
        ia, ib = np.nonzero(d < cut)
        rs += [A[ia], B[ib]]; cs += [B[ib], A[ia]]; vs += [np.full(ia.size, t)] * 2
    rowptr, colind, values = _csr_from_coo(n, np.concatenate(rs), np.concatenate(cs), np.concatenate(vs))
    layers = [np.arange(k * nring, (k + 1) * nring) for k in range(nr)]
    # Lead principal layer = one perfect 4-ring cell (no disorder).  Build a
    # 3-cell perfect tube and read the blocks off it.
    cell = _cnt_perfect_blocks(nring, t, acc)
    H00, H01 = cell
    # Left lead: device ring A0 couples axially to ring D of the lead cell next
    # to it; right lead: device ring D_last couples axially to ring A of the
    # lead cell next to it.  Lead layers are indexed away from the device.
    tauL = np.zeros((nring, 4 * nring))
    tauR = np.zeros((nring, 4 * nring))
    # coupling blocks are the D->A(next) block of H01 for the right lead
    DA = H01[3 * nring:4 * nring, 0:nring]  # rows: ring D of cell k, cols: ring A of cell k+1
    tauR[:, 0:nring] = DA  # device ring D couples to lead ring A
    tauL[:, 3 * nring:4 * nring] = DA.T  # device ring A couples to lead ring D
    # the left lead runs to -z: layer k+1 (further left) couples to layer k through H01^T
    leadL = Lead(H00=H00.copy(), H01=H01.T.copy(), tau=tauL)
    leadR = Lead(H00=H00.copy(), H01=H01.copy(), tau=tauR)
    return Device(name=f"cnt_{nring}_0_{n_cells}cells", n=n, rowptr=rowptr, colind=colind, values=values,
                  coords=coords, layers=layers, contacts=[layers[0].copy(), layers[-1].copy()],
                  leads=[leadL, leadR], transport_axis=2)


def _cnt_perfect_blocks(nring: int, t: float, acc: float) -> tuple:
    dev = None
    a = math.sqrt(3.0) * acc
    R = nring * a / (2.0 * math.pi)
    zoff, phoff = _cnt_cell_coords(nring, acc)
    m = 4 * nring
    xyz = np.zeros((2 * m, 3))
    for c in range(2):
        for r in range(4):
            phi = (np.arange(nring) + phoff[r]) * 2.0 * math.pi / nring
            sl = slice((4 * c + r) * nring, (4 * c + r + 1) * nring)
            xyz[sl, 0] = R * np.cos(phi)
            xyz[sl, 1] = R * np.sin(phi)
            xyz[sl, 2] = c * 3.0 * acc + zoff[r]
    d = np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=2)
    Hb = np.where((d < 1.1 * acc) & (d > 1e-9), t, 0.0)
    del dev
    return Hb[:m, :m].copy(), Hb[:m, m:].copy()


# Armchair ribbon cell (transport along x, one C-C bond parallel to x): four
# atom columns at x / acc = 0, 1, 1.5, 2.5, the last two shifted by half a
# period sqrt(3) acc along y; the cell repeats every 3 acc.
_AGNR_X = (0.0, 1.0, 1.5, 2.5)
_AGNR_YOFF = (0.0, 0.0, 0.5, 0.5)


def _agnr_coords(n_cells: int, ny: int, acc: float) -> np.ndarray:
    xyz = np.zeros((4 * ny * n_cells, 2))
    k = np.arange(ny)
    for c in range(n_cells):
        for r in range(4):
            sl = slice((4 * c + r) * ny, (4 * c + r + 1) * ny)
            xyz[sl, 0] = (3.0 * c + _AGNR_X[r]) * acc
            xyz[sl, 1] = (k + _AGNR_YOFF[r]) * math.sqrt(3.0) * acc
    return xyz


def agnr(n_cells: int, ny: int, *, t: float = -3.1, acc: float = 0.142, disorder: float = 0.0,
         seed: int | None = None) -> Device:
    """Armchair graphene nanoribbon, n_cells cells of four atom columns with ny
    atoms each (4 ny n_cells atoms, 2 ny dimer lines across).

    Connectivity: pairs closer than 1.1 acc (bonds only join adjacent columns).
    On-site 0 + U(-disorder, +disorder), hopping t.  Caller order is column by
    column along x.  The leads are perfect semi-infinite ribbons whose
    principal layer is one cell.
    """
    m = ny
    n = 4 * m * n_cells
    coords = _agnr_coords(n_cells, ny, acc)
    onsite = np.zeros(n)
    if disorder > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        onsite = onsite + rng.uniform(-disorder, disorder, size=n)
    rs, cs, vs = [np.arange(n)], [np.arange(n)], [onsite]
    cut = 1.1 * acc
    for col in range(4 * n_cells - 1):
        A = np.arange(col * m, (col + 1) * m)
        B = np.arange((col + 1) * m, (col + 2) * m)
        d = np.linalg.norm(coords[A][:, None, :] - coords[B][None, :, :], axis=2)
        ia, ib = np.nonzero(d < cut)
        rs += [A[ia], B[ib]]; cs += [B[ib], A[ia]]; vs += [np.full(ia.size, t)] * 2
    rowptr, colind, values = _csr_from_coo(n, np.concatenate(rs), np.concatenate(cs), np.concatenate(vs))
    layers = [np.arange(k * m, (k + 1) * m) for k in range(4 * n_cells)]
    # lead blocks read off a perfect two-cell ribbon
    two = _agnr_coords(2, ny, acc)
    d = np.linalg.norm(two[:, None, :] - two[None, :, :], axis=2)
    Hb = np.where((d < cut) & (d > 1e-9), t, 0.0)
    H00, H01 = Hb[:4 * m, :4 * m].copy(), Hb[:4 * m, 4 * m:].copy()
    DA = H01[3 * m:4 * m, 0:m]  # column 3 of a cell -> column 0 of the next cell
    tauR = np.zeros((m, 4 * m))
    tauR[:, 0:m] = DA  # the device's last column couples to column 0 of the right lead's first cell
    tauL = np.zeros((m, 4 * m))
    tauL[:, 3 * m:4 * m] = DA.T  # the device's first column couples to column 3 of the left lead's first cell
    leadL = Lead(H00=H00.copy(), H01=H01.T.copy(), tau=tauL)
    leadR = Lead(H00=H00.copy(), H01=H01.copy(), tau=tauR)
    return Device(name=f"agnr_{2 * ny}_{n_cells}cells", n=n, rowptr=rowptr, colind=colind, values=values,
                  coords=coords, layers=layers, contacts=[layers[0].copy(), layers[-1].copy()],
                  leads=[leadL, leadR], transport_axis=0)


@dataclasses.dataclass
class Transport:
    """Transport parameters of a workload (paper Sec. 4.2: Fermi levels,
    temperature, energy grid).  mu in eV, kT in eV, eta in eV."""

    energies: np.ndarray
    eta: float = 1e-6
    mu: tuple = (0.1, 0.0)
    kT: float = KB_EV * 300.0
    gamma_ph: float = 0.0  # constant phonon broadening (eV); 0 = no phonon
    mu_ph: float | None = None

    @property
    def n_e(self) -> int:
        return int(self.energies.shape[0])


def energy_grid(emin: float, emax: float, n_e: int) -> np.ndarray:
    """Inclusive uniform grid (the paper's energies are uniformly distributed
    between the end points, Sec. 4.2.1)."""
    return np.linspace(emin, emax, n_e)


def union(devices, name: str = "union", gap_nm: float = 1.0e3) -> Device:
    """Disjoint union of devices as one graph (block-diagonal H): sites of
    device d follow those of devices 0..d-1; every device keeps its contacts
    and leads; coordinates are shifted apart along the second axis by gap_nm
    per device.  ``site_offsets[d]`` marks where device d starts."""
    offs = np.concatenate([[0], np.cumsum([d.n for d in devices])]).astype(np.int64)
    rowptr = [np.zeros(1, dtype=np.int64)]
    colind, values, coords = [], [], []
    for k, d in enumerate(devices):
        rowptr.append(d.rowptr[1:].astype(np.int64) + rowptr[-1][-1])
        colind.append(d.colind.astype(np.int64) + offs[k])
        values.append(d.values)
        c = d.coords.copy()
        c[:, 1] += gap_nm * k
        coords.append(c)
    dev = Device(name=name, n=int(offs[-1]), rowptr=np.concatenate(rowptr).astype(np.int32),
                 colind=np.concatenate(colind).astype(np.int32), values=np.concatenate(values),
                 coords=np.concatenate(coords),
                 layers=[l + offs[k] for k, d in enumerate(devices) for l in d.layers],
                 contacts=[c + offs[k] for k, d in enumerate(devices) for c in d.contacts],
                 leads=[l for d in devices for l in d.leads], transport_axis=devices[0].transport_axis)
    dev.site_offsets = offs
    return dev


def uneven_batch(n_devices: int = 64, *, widths=(16, 32, 64, 96), lengths=(128, 1024), disorder: float = 0.02,
                 seed: int | None = None) -> tuple:
    """Superlattices of uneven size in one graph: width uniform over ``widths``,
    length a uniform integer in [lengths[0], lengths[1]] (PCG64 stream of
    ``seed``), onsite disorder from a seed per device.  Returns (union device,
    list of the devices)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W = rng.choice(np.asarray(widths), size=n_devices)
    L = rng.integers(lengths[0], lengths[1] + 1, size=n_devices)
    devs = [superlattice(int(l), int(w), disorder=disorder, seed=(seed or 0) * 1000 + k) for k, (l, w) in
            enumerate(zip(L, W))]
    return union(devs, name=f"uneven_{n_devices}"), devs


SEED_BASE = 1305


def workload(name: str):
    """Named workloads with the sizes used by the tests and the benchmark.

    superlattice_64x16    : 64 x 16 = 1,024 sites, 16 energies in [0, 0.5] eV
    superlattice_512x128  : 512 x 128 = 65,536 sites, disorder +-0.02 eV, 256 energies
    cnt_10_0_400          : (10,0) tube, 400 cells = 16,000 atoms, disorder +-0.1 eV,
                            phonon broadening 5 meV, 1,024 energies in [-1, 1] eV
    superlattice_256x64   : 256 x 64 = 16,384 sites, disorder +-0.02 eV, 128 energies (density gradient)
    superlattice_256x64_sp: the same device, 128 energies in [-0.6, 0.5] eV, eta = 9 meV (Schroedinger-Poisson)
    uneven_64             : 64 superlattices in one graph, widths in {16, 32, 64, 96},
                            lengths in [128, 1024], disorder +-0.02 eV, 64 energies in [0, 0.5] eV
    """
    if name == "superlattice_64x16":
        dev = superlattice(64, 16)
        tr = Transport(energies=energy_grid(0.0, 0.5, 16))
    elif name == "superlattice_512x128":
        dev = superlattice(512, 128, disorder=0.02, seed=SEED_BASE + 1)
        tr = Transport(energies=energy_grid(0.0, 0.5, 256))
    elif name == "superlattice_256x64":
        dev = superlattice(256, 64, disorder=0.02, seed=SEED_BASE + 4)
        tr = Transport(energies=energy_grid(0.0, 0.5, 128))
    elif name == "superlattice_256x64_sp":
        # the self-consistent loop: the window reaches below the flat-band edge
        # by more than the barrier height (screening pulls the barriers down by
        # up to ~0.3 eV) and eta is about the grid spacing, so that the
        # 128-point energy integral resolves the broadened one-dimensional
        # subband edges and n(U) is smooth in U
        dev = superlattice(256, 64, disorder=0.02, seed=SEED_BASE + 4)
        tr = Transport(energies=energy_grid(-0.6, 0.5, 128), eta=9e-3)
    elif name == "uneven_64":
        dev, _ = uneven_batch(64, seed=SEED_BASE + 3)
        tr = Transport(energies=energy_grid(0.0, 0.5, 64))
    elif name == "cnt_10_0_400":
        dev = cnt_zigzag(400, disorder=0.1, seed=SEED_BASE + 2)
        tr = Transport(energies=energy_grid(-1.0, 1.0, 1024), gamma_ph=5e-3, mu_ph=0.05)
    else:
        raise KeyError(name)
    return dev, tr
