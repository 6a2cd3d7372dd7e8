"""The bounded waits of the tensor-core products, made to run out on purpose
(no device fault): with a limit of one poll every wait of k_gemm_tc gives up,
its CTAs wait for their own copies and products in flight, release their
tensor memory and skip their output, and nd_fact_status reports
ND_ERR_TIMEOUT.  With the default limit restored, the next call on the same
handle matches the oracle (paper Eq. (1)-(2)) again."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, observables  # noqa: E402
from paper_1305_1070_gb300 import build, ndgf, workloads  # noqa: E402
from paper_1305_1070_gb300.solver import Solver  # noqa: E402

pytestmark = pytest.mark.gpu
TIMEOUT = 7


def test_wait_limit_runs_out_and_handle_recovers():
    build.build()
    dev = workloads.superlattice(20, 6, disorder=0.02, seed=3)
    tr = workloads.Transport(energies=np.array([0.08, 0.31]))
    ref = dense.green_diag(dev, tr)
    s = Solver(dev, tr, precision=ndgf.ND_PREC_FP32X2, leaf_size=10, delay=2, tile="tc")
    ndgf.nd_fact_set_wait_limit(s.fact, 1)
    s.step(tr.energies)
    torch.cuda.synchronize()
    with pytest.raises(ndgf.NDError) as e:
        ndgf.nd_fact_status(s.fact)
    assert e.value.status == TIMEOUT
    ndgf.nd_fact_set_wait_limit(s.fact, 0)
    for _ in range(2):
        Gr, Gl, Gg = s.step(tr.energies)
        torch.cuda.synchronize()
        assert ndgf.nd_fact_status(s.fact) == 0
        for k, g in (("Gr", Gr), ("Gl", Gl), ("Gg", Gg)):
            g = g.cpu().numpy()
            for i in range(tr.n_e):
                assert observables.rel_err(g[i], ref[k][i]) < 1e-9
    with pytest.raises(ndgf.NDError):
        ndgf.nd_fact_set_wait_limit(s.fact, -1)
