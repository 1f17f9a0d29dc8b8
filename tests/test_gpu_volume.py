"""The volume-kernel cost comparison of Sec. 5.4 on the GPU: the device DG
and ESDG volume kernels (esdg_volume_kernel) against the FP64 oracle, over
sizes that span several shared-memory column tiles (32), ragged element
counts (4 per CTA) and the largest supported matrix (256)."""

import numpy as np
import pytest

from oracle.volume import volume_dg, volume_esdg
from paper_2005_02516_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_2005_02516_gb300 import esdg
    if not os.path.exists(esdg.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()


@pytest.mark.parametrize("n,K", [(1, 1), (5, 7), (16, 13), (33, 4), (50, 9), (200, 6), (256, 5)])
@pytest.mark.parametrize("kind", ["dg", "esdg"])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
def test_device_volume_kernel_matches_oracle(n, K, kind, dtype, tol):
    from paper_2005_02516_gb300 import esdg
    Qx, Qy, u = W.volume_ratio_inputs(n, K, seed=100 + n)
    g = 1.0
    want = (volume_esdg if kind == "esdg" else volume_dg)(Qx, Qy, u, g)
    code = esdg.ESDG_VOLUME_ESDG if kind == "esdg" else esdg.ESDG_VOLUME_DG
    dev = [torch.tensor(a, dtype=dtype, device="cuda") for a in (Qx, Qy, u)]
    got = esdg.volume_kernel(code, *dev, g=g)
    torch.cuda.synchronize()
    got = got.double().cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol
