"""Failure detection without a GPU fault: a bounded wait that can never
complete gives up, the kernel records TT_ETIMEOUT in the device status word
and returns, and the context stays usable for the next decomposition."""
import numpy as np
import pytest

import oracle
from paper_2308_01480_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    import paper_2308_01480_gb300 as tt
    assert torch.cuda.is_available()
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    tt.debug_wait_timeout(ws)
    torch.cuda.synchronize()
    assert tt.device_status(ws) == tt._native.TT_ETIMEOUT
    # the context is intact: a decomposition right after succeeds
    w = W.CONFIGS[1]
    A = W.make_tensor(w)
    t = torch.from_numpy(A.astype(np.float32)).cuda()
    cores, _ = tt.decompose(t, w.ranks, w.oversample, w.q, omega_seed=w.omega_seed)
    torch.cuda.synchronize()
    assert tt.device_status(tt.decompose.last_workspace) == 0
    ref = oracle.tt_rbki(A.astype(np.float32), w.ranks, w.oversample, w.q, seed=w.omega_seed)
    assert oracle.tt_distance([c.cpu().double().numpy() for c in cores], ref) <= 1e-4
