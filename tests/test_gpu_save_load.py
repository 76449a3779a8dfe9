"""hodlr_save / hodlr_load: the loaded handle stores the matrix exactly as
the saved one -- the same formats, the same precision-rule summary, bitwise
the same exported generators and bitwise the same products (CUDA cores and
tensor cores), for fp32 and fp64 working precision and both precision
rules."""
import numpy as np
import pytest
import torch

import synth
from oracle import compress as C
from oracle import kernels as K
from oracle.abi_lists import oracle_to_abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2407_21637_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("work,per_block,eps", [("fp32", False, 1e-6), ("fp32", True, 1e-3), ("fp64", False, 1e-8)])
def test_save_load_roundtrip_is_exact(tmp_path, work, per_block, eps):
    from paper_2407_21637_gb300 import HodlrMatrix
    n, depth = 1500, 3
    tiers = ("fp64", "fp32", "bf16", "fp16", "e4m3", "e5m2")
    spec = synth.KernelSpec(K.INV_DIST, c=1e-3, diag=float(n))
    h = C.compress(synth.uniform_points_1d(n, 17), spec, n, depth, eps)
    C.assign_precisions(h, eps, work, tiers, per_block=per_block, norms="factors")
    C.store_all(h)
    ranks, U, V, D = oracle_to_abi(h)
    g = HodlrMatrix.from_factors(n, depth, ranks, U, V, D, eps=eps, work=work, tiers=tiers,
                                 per_block=per_block)
    path = tmp_path / "m.hodlr"
    g.save(path)
    g2 = HodlrMatrix.load(path)
    assert g2.n == n and g2.depth == depth and g2.work == work
    assert g2.block_tiers() == g.block_tiers()
    i1, i2 = g.info(), g2.info()
    for key in ("xi", "u_prime", "level_tier", "bytes_per_tier", "factor_bytes", "leaf_bytes", "max_rank"):
        assert i1[key] == i2[key], key
    for a, b in zip(g.export(), g2.export()):
        for x, y in zip(a, b):
            assert np.array_equal(x.view(np.int64), y.view(np.int64))
    dt = torch.float32 if work == "fp32" else torch.float64
    for R in (1, 64):
        X = torch.from_numpy(synth.rhs_normal(n, R, 40 + R)).to(dt).cuda()
        assert torch.equal(g.matvec(X), g2.matvec(X))
    g.close()
    g2.close()
