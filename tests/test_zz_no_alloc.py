"""The allocation-free batched inversion (nd_invert_c64_noalloc), for callers
that cannot allocate device memory, against the existing path that inverts a
complex64 block in complex128: nd_factor + nd_diag_green on a one-cluster
plan (the root block of the single-precision path), two calls in a row."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1305_1070_gb300 import build, ndgf, workloads  # noqa: E402

pytestmark = pytest.mark.gpu
TOL_C64 = 1e-3  # tolerance of the complex64 path in the parity tests


def test_noalloc_inverse_matches_existing_path():
    build.build()
    dev = workloads.superlattice(8, 5, disorder=0.05, seed=2)
    n, eta = dev.n, 1e-3
    plan = ndgf.nd_analyze(n, dev.rowptr, dev.colind, None, None, dev.coords, leaf_size=1000)
    assert ndgf.nd_plan_query(plan)["n_clusters"] == 1
    fact = ndgf.nd_fact_create(plan, 2, ndgf.ND_PREC_MIXED)
    H = torch.as_tensor(dev.values, device="cuda")
    Hd = torch.as_tensor(dev.dense(), device="cuda", dtype=torch.complex128)
    eye = torch.eye(n, device="cuda", dtype=torch.complex128)
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    for energies in ((0.13,), (0.41, 0.07)):  # two calls in a row, the second batched
        k = len(energies)
        E = torch.tensor(energies, device="cuda", dtype=torch.float64)
        Gr = torch.zeros(k, n, dtype=torch.complex128, device="cuda")
        ndgf.nd_factor(fact, H, None, None, E, k, eta)
        ndgf.nd_diag_green(fact, None, None, None, None, Gr, None, None)
        A = torch.stack([(e + 1j * eta) * eye - Hd for e in energies]).to(torch.complex64).contiguous()
        ndgf.nd_invert_c64_noalloc(A, n, k, cnt)
        torch.cuda.synchronize()
        assert int(cnt.item()) == 0
        for b in range(k):
            got = torch.diagonal(A[b]).cpu().numpy().astype(np.complex128)
            ref = Gr[b].cpu().numpy()
            err = np.abs(got - ref).max() / np.abs(ref).max()
            assert err <= TOL_C64, err
            # the full inverse is an inverse of the complex64 matrix
            Ab = ((energies[b] + 1j * eta) * eye - Hd).to(torch.complex64).to(torch.complex128)
            resid = (Ab @ A[b].to(torch.complex128) - eye).abs().max().item()
            assert resid <= TOL_C64, resid


def test_noalloc_near_the_cap_matches_existing_path():
    """n = 512, batch 1: batch * n * n = 2^18, the whole working space."""
    build.build()
    dev = workloads.superlattice(32, 16, disorder=0.05, seed=5)
    n, eta = dev.n, 1e-3
    assert n == 512
    plan = ndgf.nd_analyze(n, dev.rowptr, dev.colind, None, None, dev.coords, leaf_size=1000)
    assert ndgf.nd_plan_query(plan)["n_clusters"] == 1
    fact = ndgf.nd_fact_create(plan, 1, ndgf.ND_PREC_MIXED)
    H = torch.as_tensor(dev.values, device="cuda")
    Hd = torch.as_tensor(dev.dense(), device="cuda", dtype=torch.complex128)
    eye = torch.eye(n, device="cuda", dtype=torch.complex128)
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    for energy in (0.21, 0.33):  # two calls in a row over the full working space
        E = torch.tensor([energy], device="cuda", dtype=torch.float64)
        Gr = torch.zeros(1, n, dtype=torch.complex128, device="cuda")
        ndgf.nd_factor(fact, H, None, None, E, 1, eta)
        ndgf.nd_diag_green(fact, None, None, None, None, Gr, None, None)
        A = ((energy + 1j * eta) * eye - Hd).to(torch.complex64).unsqueeze(0).contiguous()
        ndgf.nd_invert_c64_noalloc(A, n, 1, cnt)
        torch.cuda.synchronize()
        assert int(cnt.item()) == 0
        got = torch.diagonal(A[0]).cpu().numpy().astype(np.complex128)
        ref = Gr[0].cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= TOL_C64, err


def test_noalloc_rejects_oversize_and_host_arrays():
    build.build()
    A = torch.zeros(1, dtype=torch.complex64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    for n, batch in ((513, 1), (1024, 1), (512, 2), (40, 200)):  # each over 2^18 elements or n > 512
        with pytest.raises(ndgf.NDError) as e:
            ndgf.nd_invert_c64_noalloc(A, n, batch, cnt)
        assert e.value.status == 1
    A_host = np.zeros((1, 8, 8), dtype=np.complex64)
    with pytest.raises(ndgf.NDError) as e:  # a host matrix is rejected before any launch
        ndgf.nd_invert_c64_noalloc(A_host, 8, 1, cnt)
    assert e.value.status == 1
    with pytest.raises(ndgf.NDError) as e:
        ndgf.nd_invert_c64_noalloc(torch.zeros(1, 8, 8, dtype=torch.complex64, device="cuda"), 8, 1,
                                   np.zeros(1, dtype=np.int32))
    assert e.value.status == 1
