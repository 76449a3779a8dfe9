"""Failure detection on the GPU without a fault: every device-side wait of
the product kernels is bounded (two seconds), records a code in the handle's
error word and lets the kernel finish.  hodlr_debug_stall_next makes the
next product's grid barrier unreachable (the host shifts the barrier target;
nothing else changes), so the waits run out; hodlr_sync_status must then
report HODLR_ETIMEOUT once, and the next products on the same handle and
context must be correct again."""
import numpy as np
import pytest
import torch

import synth
from oracle import bounds as Bd
from oracle import compress as C
from oracle import formats as F
from oracle import kernels as K
from oracle import matvec as M
from oracle.abi_lists import oracle_to_abi

pytestmark = pytest.mark.gpu

HODLR_ETIMEOUT = 4


@pytest.fixture(scope="module")
def handle():
    from paper_2407_21637_gb300 import build as B
    from paper_2407_21637_gb300 import HodlrMatrix
    B.build()
    torch.cuda.set_device(0)
    n, depth, eps = 1024, 3, 1e-6
    tiers = ("fp64", "fp32", "bf16", "fp16", "e4m3")
    spec = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
    h = C.compress(synth.uniform_points_1d(n, 5), spec, n, depth, eps)
    C.assign_precisions(h, eps, "fp32", tiers, norms="factors")
    C.store_all(h)
    ranks, U, V, D = oracle_to_abi(h)
    g = HodlrMatrix.from_factors(n, depth, ranks, U, V, D, eps=eps, work="fp32", tiers=tiers)
    yield h, g
    g.close()


def _check(h, g, R, seed):
    X = synth.rhs_normal(h.n, R, seed, np.float32)
    B = g.matvec(torch.from_numpy(X).cuda())
    g.sync_status()   # no wait gave up
    X64 = X.astype(np.float64)
    ref = M.hodlr_matvec(h, X64)
    u = F.unit_roundoff("fp32")
    tol = (Bd.gamma(M.max_chain(h), 2 * u) + 14 * u) * M.abs_product(h, X64) + u * np.abs(ref)
    assert np.all(np.abs(B.cpu().numpy().astype(np.float64) - ref) <= tol)


@pytest.mark.parametrize("R", [1, 64])
def test_barrier_timeout_is_reported_and_the_context_stays_usable(handle, R):
    from paper_2407_21637_gb300 import HodlrError
    h, g = handle
    _check(h, g, R, 1)
    X = torch.from_numpy(synth.rhs_normal(h.n, R, 2, np.float32)).cuda()
    g.debug_stall_next()
    g.matvec(X)
    with pytest.raises(HodlrError) as e:
        g.sync_status()
    assert e.value.status == HODLR_ETIMEOUT
    g.sync_status()   # reported once, then clear
    _check(h, g, R, 3)
