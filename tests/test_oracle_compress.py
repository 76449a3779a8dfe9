"""Pins for oracle.compress: known-rank kernels, exact reconstruction,
Lemma 2.4, eq. (3.5), Thm 3.1 and the precision rule of Algorithm 3.2."""
import math

import numpy as np
import pytest

import synth
from oracle import bounds as Bd
from oracle import compress as C
from oracle import formats as F
from oracle import kernels as K
from oracle import matvec as M


def _pts(n, seed=11):
    return synth.uniform_points_1d(n, seed)


@pytest.mark.parametrize("name,f,rank", [
    ("sq_dist", lambda x, y: (x - y) ** 2, 3),
    ("cos", lambda x, y: np.cos(7.0 * (x - y)), 2),
    ("poly2", lambda x, y: (1.0 + x * y) ** 2, 3),
])
def test_separable_kernels_have_exact_rank(name, f, rank):
    n, depth = 512, 3
    x = _pts(n)[:, 0]
    A = f(x[:, None], x[None, :])
    h = C.compress(None, None, n, depth, eps=1e-12, A=A)
    for k in range(1, depth + 1):
        for i in range(1 << k):
            assert h.rank(k, i) == rank, (k, i, h.rank(k, i))
    At = M.assemble(h, stored=False)
    assert np.linalg.norm(At - A) <= 1e-13 * np.linalg.norm(A)


def test_eps_zero_reconstructs_exactly():
    n, depth = 256, 3
    rng = np.random.default_rng(5)
    A = rng.standard_normal((n, n))
    h = C.compress(None, None, n, depth, eps=0.0, A=A)
    for k in range(1, depth + 1):
        for i in range(1 << k):
            assert h.rank(k, i) == n >> k          # full rank of a random block
    assert np.linalg.norm(M.assemble(h, stored=False) - A) <= 1e-13 * np.linalg.norm(A)


def test_truncation_rank_is_minimal():
    rng = np.random.default_rng(6)
    for trial in range(20):
        m = 40
        Q1, _ = np.linalg.qr(rng.standard_normal((m, m)))
        Q2, _ = np.linalg.qr(rng.standard_normal((m, m)))
        s = np.sort(np.exp(rng.uniform(-30, 0, m)))[::-1]
        A = (Q1 * s) @ Q2.T
        eps = 10.0 ** rng.uniform(-10, -1)
        U, V, sv = C.truncated_svd(A, eps)
        r = U.shape[1]
        tail = lambda q: math.sqrt(float(np.sum(sv[q:] ** 2)))
        tot = math.sqrt(float(np.sum(sv ** 2)))
        assert tail(r) <= eps * tot
        if r > 0:
            assert tail(r - 1) > eps * tot
        assert np.allclose(U.T @ U, np.eye(r), atol=1e-13)


KERNELS = [
    ("inv_dist", synth.KernelSpec(K.INV_DIST, c=1e-3, diag=512.0)),
    ("gauss", synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)),
    ("log", synth.KernelSpec(K.LOG, c=1e-4, diag=512.0)),
]


@pytest.mark.parametrize("kname,spec", KERNELS)
@pytest.mark.parametrize("eps", [1e-2, 1e-5, 1e-9])
def test_lemma_2_4_every_level(kname, spec, eps):
    """||H~_ii^(k) - H_ii^(k)||_F <= eps ||H_ii^(k)||_F for every level k."""
    n, depth = 512, 4
    pts = _pts(n)
    A = K.kernel_matrix(pts, spec)
    h = C.compress(pts, spec, n, depth, eps)
    E = M.assemble(h, stored=False) - A
    for k in range(depth + 1):
        for (s, m) in h.levels[k]:
            blk = slice(s, s + m)
            assert np.linalg.norm(E[blk, blk]) <= eps * np.linalg.norm(A[blk, blk]) * (1 + 1e-12) + 1e-300


@pytest.mark.parametrize("fmt", ["fp32", "bf16", "fp16", "e4m3", "e5m2"])
def test_eq_3_5_per_block_storage(fmt):
    """||H~_ij - H^_ij||_F <= (2 + sqrt(p) u) u ||H~_ij||_F in every block."""
    n, depth = 512, 4
    pts = _pts(n)
    spec = KERNELS[0][1]
    h = C.compress(pts, spec, n, depth, 1e-6)
    for k in range(1, depth + 1):
        h.tier[k] = [fmt] * (1 << k)
    h.work = "fp64"
    C.store_all(h)
    u = F.unit_roundoff(fmt)
    for k in range(1, depth + 1):
        for i in range(1 << k):
            Ht = h.U[k][i] @ h.V[k][i ^ 1].T
            Hh = h.Uh[k][i] @ h.Vh[k][i ^ 1].T
            p = h.rank(k, i)
            assert np.linalg.norm(Ht - Hh) <= Bd.block_storage_bound(p, u) * np.linalg.norm(Ht)


@pytest.mark.parametrize("kname,spec", KERNELS)
@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6])
def test_theorem_3_1_global_error(kname, spec, eps):
    n, depth = 1024, 5
    pts = _pts(n)
    A = K.kernel_matrix(pts, spec)
    h = C.adaptive_hodlr(pts, spec, n, depth, eps, work="fp64",
                         tiers=("fp64", "fp32", "bf16", "fp16", "e4m3", "e5m2"), A=A)
    err = np.linalg.norm(M.assemble(h) - A)
    assert err <= Bd.global_bound_rule(eps, depth) * np.linalg.norm(A)
    # the general form with the chosen u_k
    uk = [0.0] + [F.unit_roundoff(h.tier[k][0]) for k in range(1, depth + 1)]
    assert err <= Bd.global_bound_general(eps, h.xi, uk) * np.linalg.norm(A) * 1.01


def test_large_eps_uses_low_precision():
    """Larger eps admits lower precisions (Sect. 3.2); tiers get no less
    precise as eps grows."""
    n, depth = 1024, 5
    pts = _pts(n)
    spec = KERNELS[1][1]
    A = K.kernel_matrix(pts, spec)
    tiers_by_eps = []
    for eps in (1e-8, 1e-4, 1e-1):
        h = C.adaptive_hodlr(pts, spec, n, depth, eps, work="fp64",
                             tiers=("fp64", "fp32", "bf16", "fp16", "e5m2"), A=A)
        tiers_by_eps.append([F.unit_roundoff(h.tier[k][0]) for k in range(1, depth + 1)])
    assert all(a <= b for a, b in zip(tiers_by_eps[0], tiers_by_eps[1]))
    assert all(a <= b for a, b in zip(tiers_by_eps[1], tiers_by_eps[2]))
    assert max(tiers_by_eps[2]) >= F.unit_roundoff("bf16")


def _with_norms(level_norm2, n=64, depth=2):
    """A tree whose level-k blocks all have ||H_ij||_F^2 = level_norm2[k] and
    ||H||_F^2 = 1 (only the norms enter the precision rule)."""
    h = C.Hodlr(n, depth)
    h.block_norm2 = [[]] + [[level_norm2[k]] * (1 << k) for k in range(1, depth + 1)]
    h.norm2_all = 1.0
    return h


def test_precision_rule_hand_built_boundaries():
    """u'_k = eps / (2^{k/2} xi_k) for prescribed xi_k and the choice of the
    largest u* <= u'_k."""
    eps = 2.0 ** -12
    # level 1: xi = 1/4 -> u' = 2^-12 * 4 / sqrt(2) = 2^-10.5 -> fp16 (2^-11 <= u' < 2^-8)
    # level 2: xi = 1/64 -> u' = 2^-12 * 64 / 2 = 2^-7 -> bf16 (2^-8)
    h = _with_norms({1: 1.0 / 16.0, 2: 1.0 / 4096.0})
    C.assign_precisions(h, eps, "fp64", ("fp64", "fp32", "fp16", "bf16", "e5m2"))
    assert h.xi[1] == 0.25 and h.xi[2] == 1.0 / 64.0
    assert h.u_prime[1] == pytest.approx(2.0 ** -10.5, rel=1e-15)
    assert h.u_prime[2] == 2.0 ** -7
    assert h.tier[1] == ["fp16", "fp16"]
    assert h.tier[2] == ["bf16"] * 4
    # without fp16 and bf16, both levels fall to the next more precise format
    C.assign_precisions(h, eps, "fp64", ("fp64", "fp32", "e5m2"))
    assert h.tier[1][0] == "fp32" and h.tier[2][0] == "fp32"
    # empty admissible set: the most precise available format is taken
    C.assign_precisions(h, 1e-12, "bf16", ("bf16", "e5m2"))
    assert h.tier[1][0] == "bf16" and h.tier[2][0] == "bf16"
    # the working precision u itself is always in the admissible set
    C.assign_precisions(h, eps, "fp32", ("e5m2",))
    assert h.tier[1][0] == "fp32"


def test_precision_rule_exact_tie_even_level():
    """k = 2 makes 2^{k/2} exact; xi = 1/4 and eps = 2^-12 give u' = 2^-11 =
    u(fp16) exactly, which is admissible (<=)."""
    h = _with_norms({1: 0.0, 2: 1.0 / 16.0})
    C.assign_precisions(h, 2.0 ** -12, "fp64", ("fp64", "fp32", "fp16", "bf16"))
    assert h.u_prime[2] == 2.0 ** -11
    assert h.tier[2][0] == "fp16"
    # a hair below the tie, fp16 is no longer admissible
    C.assign_precisions(h, 2.0 ** -12 * (1 - 2.0 ** -40), "fp64", ("fp64", "fp32", "fp16", "bf16"))
    assert h.tier[2][0] == "fp32"
    # level 1 has zero blocks: xi = 0 -> u' = inf -> the least precise format
    assert h.tier[1][0] == "bf16"


def test_per_block_rule_is_no_more_precise_than_per_level():
    n, depth = 512, 4
    pts = _pts(n)
    spec = KERNELS[0][1]
    A = K.kernel_matrix(pts, spec)
    hl = C.adaptive_hodlr(pts, spec, n, depth, 1e-3, tiers=("fp64", "fp32", "bf16", "fp16", "e4m3"), A=A)
    hb = C.adaptive_hodlr(pts, spec, n, depth, 1e-3, tiers=("fp64", "fp32", "bf16", "fp16", "e4m3"),
                          per_block=True, A=A)
    for k in range(1, depth + 1):
        for i in range(1 << k):
            assert F.unit_roundoff(hb.tier[k][i]) >= F.unit_roundoff(hl.tier[k][i])
    err = np.linalg.norm(M.assemble(hb) - A)
    assert err <= Bd.global_bound_rule(1e-3, depth) * np.linalg.norm(A)


def test_factor_norms_choose_same_tiers():
    """xi from the fp64 factors (the estimate used at import) and from H
    itself pick the same formats away from tier boundaries."""
    n, depth = 1024, 5
    pts = _pts(n)
    for spec in (KERNELS[0][1], KERNELS[1][1]):
        A = K.kernel_matrix(pts, spec)
        for eps in (1e-2, 1e-4, 1e-6):
            h1 = C.adaptive_hodlr(pts, spec, n, depth, eps, tiers=("fp64", "fp32", "bf16", "fp16", "e4m3"), A=A)
            h2 = C.compress(pts, spec, n, depth, eps, A=A)
            C.assign_precisions(h2, eps, "fp64", ("fp64", "fp32", "bf16", "fp16", "e4m3"), norms="factors")
            for k in range(1, depth + 1):
                ratio = h1.u_prime[k] / h2.u_prime[k]
                assert abs(ratio - 1) < 2 * eps + 1e-12
                if h1.tier[k] != h2.tier[k]:
                    up = h1.u_prime[k]
                    near = [f for f in F.FORMATS if abs(F.unit_roundoff(f) / up - 1) < 2 * eps]
                    assert near, (k, h1.tier[k], h2.tier[k])


def test_planted_dropped_sigma_is_caught():
    """Storing V without Sigma (a plausible slip) breaks Lemma 2.4."""
    n, depth = 256, 3
    pts = _pts(n)
    spec = KERNELS[0][1]
    A = K.kernel_matrix(pts, spec)
    h = C.compress(pts, spec, n, depth, 1e-6)
    for k in range(1, depth + 1):
        for j in range(1 << k):
            v = h.V[k][j]
            h.V[k][j] = v / np.maximum(np.linalg.norm(v, axis=0), 1e-300)
    E = M.assemble(h, stored=False) - A
    assert np.linalg.norm(E) > 1e-6 * np.linalg.norm(A)
