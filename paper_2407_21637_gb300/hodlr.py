"""Python handle around the C ABI (argument marshalling only).

Every step of the product runs in libhodlr's kernels; this module converts
Python/torch arguments to pointers and sizes, and raises on a non-OK status.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np
import torch

from ._lib import PREC, PREC_NAME, BuildOpts, Info, Kernel, Opts, SolveStats, check, load

_TORCH_DTYPE = {"fp64": torch.float64, "fp32": torch.float32}


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr_array(mats: Sequence):
    """Array of double* for a list of C-contiguous float64 numpy arrays (None -> NULL)."""
    arr = (ctypes.POINTER(ctypes.c_double) * max(len(mats), 1))()
    keep = []
    for i, m in enumerate(mats):
        if m is None or m.size == 0:
            arr[i] = ctypes.POINTER(ctypes.c_double)()
            continue
        a = np.ascontiguousarray(m, dtype=np.float64)
        keep.append(a)
        arr[i] = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return arr, keep


class HodlrMatrix:
    """A stored adaptive-precision HODLR matrix on the current CUDA device."""

    def __init__(self, handle: ctypes.c_void_p, n: int, depth: int, work: str):
        self._h = handle
        self.n, self.depth, self.work = n, depth, work
        self.dtype = _TORCH_DTYPE[work]

    # ---- construction -------------------------------------------------
    @classmethod
    def from_factors(cls, n: int, depth: int, ranks: Sequence[int], U: Sequence, V: Sequence,
                     D: Sequence, eps: float, work: str = "fp32",
                     tiers: Sequence[str] = ("fp64", "fp32", "bf16", "fp16", "e4m3"),
                     per_block: bool = False, max_nrhs: int = 64, stream=None) -> "HodlrMatrix":
        """hodlr_import: per-node lists in level order (level 1, then 2, ...):
        ``ranks[q]`` = rank of block (i, i^1); ``U[q]`` (m_i x rank) and
        ``V[q]`` (m_i x rank of the sibling's block); ``D`` per leaf."""
        lib = load()
        nn = (1 << (depth + 1)) - 2
        if len(ranks) != nn or len(U) != nn or len(V) != nn or len(D) != (1 << depth):
            raise ValueError("per-node lists must have 2^(depth+1)-2 entries and D 2^depth")
        r = (ctypes.c_int32 * max(nn, 1))(*[int(x) for x in ranks])
        pu, ku = _dptr_array(U)
        pv, kv = _dptr_array(V)
        pd, kd = _dptr_array(D)
        mask = 0
        for t in tiers:
            mask |= 1 << PREC[t]
        opts = Opts(eps=float(eps), work=PREC[work], tier_mask=mask, per_block=int(per_block),
                    max_nrhs=int(max_nrhs))
        h = ctypes.c_void_p()
        check(lib.hodlr_import(n, depth, r, pu, pv, pd, ctypes.byref(opts), _stream_ptr(stream),
                               ctypes.byref(h)), "hodlr_import")
        del ku, kv, kd
        return cls(h, n, depth, work)

    @classmethod
    def build(cls, points: torch.Tensor, kind: int, depth: int, eps: float, c: float = 0.0,
              len2: float = 1.0, diag: float = 0.0, work: str = "fp32",
              tiers: Sequence[str] = ("fp64", "fp32", "bf16", "fp16", "e4m3"),
              per_block: bool = False, max_nrhs: int = 64, sketch: int = 0, max_sketch: int = 0,
              seed: int = 0, stream=None, allow_short: bool = False,
              node_sketch: Sequence[int] | None = None) -> "HodlrMatrix":
        """hodlr_build: compress the kernel matrix of ``points`` ((n, dim) fp64
        CUDA tensor, tree order) on the GPU (Algorithm 3.2 with a randomized
        range finder) and store it in the adaptive-precision format."""
        lib = load()
        pts = points if points.dim() == 2 else points.view(-1, 1)
        if pts.dtype != torch.float64 or not pts.is_cuda:
            raise ValueError("points must be a float64 CUDA tensor")
        pts = pts.contiguous()
        n, dim = pts.shape
        kern = Kernel(kind=int(kind), dim=int(dim), c=float(c), len2=float(len2), diag=float(diag))
        mask = 0
        for t in tiers:
            mask |= 1 << PREC[t]
        opts = Opts(eps=float(eps), work=PREC[work], tier_mask=mask, per_block=int(per_block),
                    max_nrhs=int(max_nrhs))
        bo = BuildOpts(sketch=int(sketch), max_sketch=int(max_sketch), seed=int(seed))
        if node_sketch is not None:
            ns = np.ascontiguousarray(np.asarray(node_sketch, dtype=np.int32))
            if ns.size != (1 << (depth + 1)) - 2:
                raise ValueError("node_sketch needs one entry per node (2^(depth+1) - 2)")
            bo.node_sketch = ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            bo._keep = ns   # the array must outlive the call
        h = ctypes.c_void_p()
        st = lib.hodlr_build(n, depth, ctypes.byref(kern), ctypes.c_void_p(pts.data_ptr()),
                             ctypes.byref(opts), ctypes.byref(bo), _stream_ptr(stream), ctypes.byref(h))
        if st == 7 and allow_short and h.value:
            return cls(h, n, depth, work)
        check(st, "hodlr_build")
        return cls(h, n, depth, work)

    # ---- products -----------------------------------------------------
    def matvec(self, X: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """B = H X on the device (hodlr_matvec).  X: (n,) or (n, R) CUDA tensor of
        the working dtype, rows contiguous (stride(1) == 1)."""
        vec = X.dim() == 1
        X2 = X.view(-1, 1) if vec else X
        if X2.dtype != self.dtype or not X2.is_cuda or X2.shape[0] != self.n or X2.stride(1) != 1:
            raise ValueError("X must be a CUDA (n, R) tensor of the working dtype with unit column stride")
        R = X2.shape[1]
        if out is None:
            out = torch.empty((self.n, R), dtype=self.dtype, device=X2.device)
        B2 = out.view(-1, 1) if out.dim() == 1 else out
        if B2.shape != (self.n, R) or B2.dtype != self.dtype or B2.stride(1) != 1:
            raise ValueError("out has the wrong shape/dtype/layout")
        ldx = X2.stride(0) if R > 1 else max(X2.stride(0), 1)
        ldb = B2.stride(0) if R > 1 else max(B2.stride(0), 1)
        check(load().hodlr_matvec(self._h, R, ctypes.c_void_p(X2.data_ptr()), ldx,
                                  ctypes.c_void_p(B2.data_ptr()), ldb, PREC[self.work],
                                  _stream_ptr(stream)), "hodlr_matvec")
        return out.view(-1) if vec and out.dim() == 2 else out

    def save(self, path: str, stream=None):
        """hodlr_save: write the stored matrix (exactly) to a file."""
        check(load().hodlr_save(self._h, str(path).encode(), _stream_ptr(stream)), "hodlr_save")

    @classmethod
    def load(cls, path: str, stream=None) -> "HodlrMatrix":
        """hodlr_load: a handle stored exactly as the saved one."""
        lib = load()
        h = ctypes.c_void_p()
        check(lib.hodlr_load(str(path).encode(), _stream_ptr(stream), ctypes.byref(h)), "hodlr_load")
        inf = Info()
        check(lib.hodlr_info(h, ctypes.byref(inf)), "hodlr_info")
        return cls(h, inf.n, inf.depth, PREC_NAME[inf.work])

    def sync_status(self, stream=None):
        """hodlr_sync_status: wait for the stream; raise HodlrError
        (HODLR_ETIMEOUT) when a device-side wait of this handle gave up."""
        check(load().hodlr_sync_status(self._h, _stream_ptr(stream)), "hodlr_sync_status")

    def debug_stall_next(self):
        """hodlr_debug_stall_next: the next matvec's grid barrier waits run
        out (a test of the timeout path)."""
        check(load().hodlr_debug_stall_next(self._h), "hodlr_debug_stall_next")

    # ---- inspection ---------------------------------------------------
    def info(self) -> dict:
        inf = Info()
        check(load().hodlr_info(self._h, ctypes.byref(inf)), "hodlr_info")
        d = self.depth
        return {
            "n": inf.n, "depth": inf.depth, "work": PREC_NAME[inf.work], "per_block": inf.per_block,
            "max_rank": inf.max_rank, "n_blocks": inf.n_blocks,
            "factor_bytes": inf.factor_bytes, "leaf_bytes": inf.leaf_bytes,
            "u_bytes": inf.u_bytes, "v_bytes": inf.v_bytes,
            "scale_bytes": inf.scale_bytes, "device_bytes": inf.device_bytes,
            "bytes_per_tier": {PREC_NAME[p]: inf.bytes_per_tier[p] for p in range(6)},
            "norm2_all": inf.norm2_all,
            "xi": [inf.xi[k] for k in range(d + 1)],
            "u_prime": [inf.u_prime[k] for k in range(d + 1)],
            "level_tier": [PREC_NAME.get(inf.level_tier[k], "?") if k else None for k in range(d + 1)],
        }

    def profile(self, enable: bool = True):
        """hodlr_profile: time each kernel of the following products with CUDA events."""
        check(load().hodlr_profile(self._h, int(enable)), "hodlr_profile")

    def profile_read(self):
        """hodlr_profile_read: device ms of the two kernels of the last profiled
        product (tensor-core kernel, product kernel), or (product kernel, 0)."""
        ms = (ctypes.c_float * 2)()
        check(load().hodlr_profile_read(self._h, ms, 2), "hodlr_profile_read")
        return float(ms[0]), float(ms[1])

    def block_tiers(self):
        nn = (1 << (self.depth + 1)) - 2
        t = (ctypes.c_int32 * max(nn, 1))()
        r = (ctypes.c_int32 * max(nn, 1))()
        check(load().hodlr_block_tiers(self._h, t, r), "hodlr_block_tiers")
        return [PREC_NAME[t[q]] for q in range(nn)], [r[q] for q in range(nn)]

    def build_stats(self):
        """hodlr_build_stats: (rounds, blocks redone, sketch columns summed over rounds)."""
        r, d = ctypes.c_int32(), ctypes.c_int32()
        c = ctypes.c_int64()
        check(load().hodlr_build_stats(self._h, ctypes.byref(r), ctypes.byref(d), ctypes.byref(c)),
              "hodlr_build_stats")
        return r.value, d.value, c.value

    def node_sizes(self):
        """The cluster tree from the library (hodlr_node_sizes): levels[k][i] =
        (first row, rows) of node (k, i); levels[0] = [(0, n)]."""
        nn = (1 << (self.depth + 1)) - 2
        r0 = (ctypes.c_int32 * max(nn, 1))()
        mm = (ctypes.c_int32 * max(nn, 1))()
        check(load().hodlr_node_sizes(self._h, r0, mm), "hodlr_node_sizes")
        levels = [[(0, self.n)]]
        for k in range(1, self.depth + 1):
            levels.append([(r0[(1 << k) - 2 + i], mm[(1 << k) - 2 + i]) for i in range(1 << k)])
        return levels

    def export(self, stream=None):
        """Stored generators decoded to fp64 (hodlr_export): (U, V, D) lists."""
        lv = self.node_sizes()
        _tiers, ranks = self.block_tiers()
        U, V = [], []
        for k in range(1, self.depth + 1):
            for i, (_s, m) in enumerate(lv[k]):
                q = (1 << k) - 2 + i
                qs = (1 << k) - 2 + (i ^ 1)
                U.append(np.zeros((m, ranks[q])))
                V.append(np.zeros((m, ranks[qs])))
        D = [np.zeros((m, m)) for (_s, m) in lv[self.depth]]
        pu, _ = _dptr_array(U)
        pv, _ = _dptr_array(V)
        pd, _ = _dptr_array(D)
        check(load().hodlr_export(self._h, pu, pv, pd, _stream_ptr(stream)), "hodlr_export")
        return U, V, D

    # ---- HODLR LU and solves (Sect. 3.4) -----------------------------------
    def lu(self, eps_lu: float, stream=None):
        """hodlr_lu: HODLR LU (Algorithm 3.4) with Schur complements truncated
        to eps_lu, kept in the handle."""
        check(load().hodlr_lu(self._h, float(eps_lu), _stream_ptr(stream)), "hodlr_lu")

    @staticmethod
    def _cols(A: torch.Tensor, n: int) -> torch.Tensor:
        A2 = A.view(-1, 1) if A.dim() == 1 else A
        if A2.dtype != torch.float64 or not A2.is_cuda or A2.shape[0] != n or A2.stride(1) != 1:
            raise ValueError("expected a CUDA fp64 (n, R) tensor with unit column stride")
        return A2

    def lu_solve(self, B: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """hodlr_lu_solve: X = U^{-1} L^{-1} B."""
        B2 = self._cols(B, self.n)
        X = out if out is not None else torch.empty_like(B2)
        X2 = self._cols(X, self.n)
        R = B2.shape[1]
        check(load().hodlr_lu_solve(self._h, R, ctypes.c_void_p(B2.data_ptr()), max(B2.stride(0), R),
                                    ctypes.c_void_p(X2.data_ptr()), max(X2.stride(0), R), _stream_ptr(stream)),
              "hodlr_lu_solve")
        return X.view(-1) if B.dim() == 1 else X

    def solve(self, B: torch.Tensor, tol: float = 1e-12, max_it: int = 10, out: torch.Tensor | None = None,
              stream=None):
        """hodlr_solve (GMRES-based iterative refinement): returns (X, status,
        stats) where stats = {iterations, gmres_steps, backward_error};
        status is HODLR_OK or HODLR_EACCURACY (tol not reached), other
        statuses raise."""
        B2 = self._cols(B, self.n)
        X = out if out is not None else torch.empty_like(B2)
        X2 = self._cols(X, self.n)
        R = B2.shape[1]
        st = SolveStats()
        rc = load().hodlr_solve(self._h, R, ctypes.c_void_p(B2.data_ptr()), max(B2.stride(0), R),
                                ctypes.c_void_p(X2.data_ptr()), max(X2.stride(0), R), float(tol), int(max_it),
                                ctypes.byref(st), _stream_ptr(stream))
        if rc not in (0, 7):
            check(rc, "hodlr_solve")
        stats = {"iterations": st.iterations, "gmres_steps": st.gmres_steps, "backward_error": st.backward_error}
        return (X.view(-1) if B.dim() == 1 else X), rc, stats

    def lu_export(self, stream=None):
        """hodlr_lu_export: (ranks_u, ranks_v, U, V, D) of the factors."""
        nn = (1 << (self.depth + 1)) - 2
        ru = (ctypes.c_int32 * max(nn, 1))()
        rv = (ctypes.c_int32 * max(nn, 1))()
        lib = load()
        null = ctypes.POINTER(ctypes.POINTER(ctypes.c_double))()
        check(lib.hodlr_lu_export(self._h, ru, rv, null, null, null, _stream_ptr(stream)), "hodlr_lu_export")
        lv = self.node_sizes()
        U, V = [], []
        for k in range(1, self.depth + 1):
            for i, (_s, m) in enumerate(lv[k]):
                q = (1 << k) - 2 + i
                U.append(np.zeros((m, ru[q])))
                V.append(np.zeros((m, rv[q])))
        D = [np.zeros((m, m)) for (_s, m) in lv[self.depth]]
        pu, _ = _dptr_array(U)
        pv, _ = _dptr_array(V)
        pd, _ = _dptr_array(D)
        check(lib.hodlr_lu_export(self._h, ru, rv, pu, pv, pd, _stream_ptr(stream)), "hodlr_lu_export")
        return [ru[q] for q in range(nn)], [rv[q] for q in range(nn)], U, V, D

    def close(self):
        if self._h:
            load().hodlr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RankPredictor:
    """The block-rank predictor (hodlr_mlp_*): fp32 master parameters and
    their fp16 copy on the device, Adam moments, features of a kernel
    matrix's blocks, training and first-sketch sizes for hodlr_build."""

    N_IN = 11

    def __init__(self, params: np.ndarray | None = None, seed: int = 0, device=None):
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.P = int(load().hodlr_mlp_num_params())
        if params is None:
            params = self.init_params(seed)
        p = np.asarray(params, dtype=np.float32)
        if p.size != self.P:
            raise ValueError(f"expected {self.P} parameters")
        self.w32 = torch.from_numpy(p.copy()).to(dev)
        self.w16 = self.w32.half()
        self.m = torch.zeros_like(self.w32)
        self.v = torch.zeros_like(self.w32)
        self.step = 0
        self.device = dev

    def init_params(self, seed: int) -> np.ndarray:
        """He-style initialization of the layout: weights ~ N(0, 2 / fan_in), biases 0."""
        rng = np.random.default_rng(seed)
        parts = []
        for shape in ((64, 11), (64,), (64, 64), (64,), (64, 64), (64,), (1, 64), (1,)):
            parts.append(rng.standard_normal(shape).ravel() * np.sqrt(2.0 / shape[1]) if len(shape) == 2
                         else np.zeros(shape))
        return np.concatenate(parts)

    @staticmethod
    def _p(t):
        return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p()

    def features(self, points: torch.Tensor, kind: int, depth: int, eps: float, c: float = 0.0,
                 len2: float = 1.0, diag: float = 0.0, stream=None) -> torch.Tensor:
        pts = (points if points.dim() == 2 else points.view(-1, 1)).contiguous()
        n, dim = pts.shape
        feat = torch.empty(((1 << (depth + 1)) - 2, self.N_IN), dtype=torch.float32, device=pts.device)
        kern = Kernel(kind=int(kind), dim=int(dim), c=float(c), len2=float(len2), diag=float(diag))
        check(load().hodlr_mlp_features(ctypes.byref(kern), self._p(pts), n, depth, float(eps), self._p(feat),
                                        _stream_ptr(stream)), "hodlr_mlp_features")
        return feat

    def forward(self, X: torch.Tensor, act: bool = False, stream=None):
        X = X.contiguous()
        S = X.shape[0]
        y = torch.empty(S, dtype=torch.float32, device=X.device)
        a = torch.empty((S, 192), dtype=torch.float32, device=X.device) if act else None
        check(load().hodlr_mlp_forward(self._p(self.w16), S, self._p(X), self._p(y), self._p(a), _stream_ptr(stream)),
              "hodlr_mlp_forward")
        return (y, a) if act else y

    def gradient(self, X: torch.Tensor, t: torch.Tensor, stream=None):
        """(loss, grad) of the mean squared error over the samples."""
        X = X.contiguous()
        t = t.contiguous().float()
        S = X.shape[0]
        y, a = self.forward(X, act=True, stream=stream)
        dy = torch.empty_like(y)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        lib = load()
        check(lib.hodlr_mlp_loss(S, self._p(y), self._p(t), self._p(dy), self._p(loss), _stream_ptr(stream)),
              "hodlr_mlp_loss")
        grad = torch.empty_like(self.w32)
        work = torch.empty((S, 192), dtype=torch.float32, device=X.device)
        check(lib.hodlr_mlp_backward(self._p(self.w16), S, self._p(X), self._p(a), self._p(dy), self._p(grad),
                                     self._p(work), _stream_ptr(stream)), "hodlr_mlp_backward")
        return loss, grad

    def adam(self, grad: torch.Tensor, lr: float, stream=None):
        self.step += 1
        check(load().hodlr_mlp_adam(self._p(self.w32), self._p(self.w16), self._p(self.m), self._p(self.v),
                                    self._p(grad), self.step, float(lr), _stream_ptr(stream)), "hodlr_mlp_adam")

    def train(self, X: torch.Tensor, t: torch.Tensor, epochs: int = 200, lr: float = 3e-3, stream=None):
        """Full-batch Adam; returns the loss before each step (host floats)."""
        losses = []
        for _ in range(epochs):
            loss, grad = self.gradient(X, t, stream=stream)
            self.adam(grad, lr, stream=stream)
            losses.append(loss)
        return [float(v.item()) for v in losses]

    @staticmethod
    def sketch_sizes(y, smin: int = 16, smax: int = 64, over: int = 8) -> np.ndarray:
        """First sketch per block: the predicted rank 2^y - 1 plus `over`
        columns, rounded up to a multiple of 8, in [smin, smax] (smin = the
        construction's default first sketch, so the prediction only raises
        it: a round of the range finder costs about the same for any sketch
        up to 64 columns, while a block whose sketch falls short costs another
        round)."""
        y = y.detach().cpu().numpy().astype(np.float64) if isinstance(y, torch.Tensor) else np.asarray(y, np.float64)
        r = np.maximum(np.exp2(y) - 1.0, 0.0)
        return np.clip(np.ceil((r + over) / 8.0) * 8.0, smin, smax).astype(np.int32)


class HodlrBatch:
    """A planned batch of products B_i = H_i X_i in one launch
    (hodlr_batch_create / _run / _tune / _destroy).  Keeps the handles and
    the X/B tensors alive for its own lifetime."""

    def __init__(self, mats: Sequence["HodlrMatrix"], Xs: Sequence[torch.Tensor], Bs: Sequence[torch.Tensor]):
        if not (len(mats) == len(Xs) == len(Bs)) or not mats:
            raise ValueError("one X and one B per matrix")
        work = mats[0].work
        self._keep = (list(mats), list(Xs), list(Bs))
        cnt = len(mats)
        hs = (ctypes.c_void_p * cnt)(*[m._h for m in mats])
        nr = (ctypes.c_int32 * cnt)()
        xp = (ctypes.c_void_p * cnt)()
        bp = (ctypes.c_void_p * cnt)()
        lx = (ctypes.c_int64 * cnt)()
        lb = (ctypes.c_int64 * cnt)()
        for i, (m, X, B) in enumerate(zip(mats, Xs, Bs)):
            if X.dim() != 2 or B.dim() != 2 or X.stride(1) != 1 or B.stride(1) != 1 or X.shape != B.shape:
                raise ValueError("X and B must be (n, R) tensors with unit column stride")
            if X.dtype != m.dtype or B.dtype != m.dtype or not X.is_cuda or not B.is_cuda or X.shape[0] != m.n:
                raise ValueError("X and B must be CUDA tensors of the matrix's working dtype with n rows")
            nr[i] = X.shape[1]
            xp[i] = X.data_ptr()
            bp[i] = B.data_ptr()
            lx[i] = X.stride(0)
            lb[i] = B.stride(0)
        self._b = ctypes.c_void_p()
        check(load().hodlr_batch_create(cnt, hs, nr, xp, lx, bp, lb, PREC[work], ctypes.byref(self._b)),
              "hodlr_batch_create")

    def run(self, threads: int = 0, stream=None):
        check(load().hodlr_batch_run(self._b, int(threads), _stream_ptr(stream)), "hodlr_batch_run")

    def tune(self, stream=None):
        th = ctypes.c_int32()
        ms = ctypes.c_float()
        check(load().hodlr_batch_tune(self._b, _stream_ptr(stream), ctypes.byref(th), ctypes.byref(ms)),
              "hodlr_batch_tune")
        return th.value, ms.value

    def close(self):
        if self._b:
            load().hodlr_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HodlrPart:
    """Part j of a product partitioned at tree level g (hodlr_part_*): the
    rows of node (g, j).  ``partial(X_j, yred)`` fills ``yred`` (the levels
    1..g of V^T X over the part's rows); the caller sums ``yred`` over the
    2^g parts (e.g. ``torch.distributed.all_reduce``); ``finish(X_j, yred)``
    returns the part's rows of H X.  Keeps the matrix alive."""

    def __init__(self, matrix: "HodlrMatrix", g: int, j: int, nrhs: int):
        self._m = matrix
        self.nrhs = int(nrhs)
        self._p = ctypes.c_void_p()
        check(load().hodlr_part_create(matrix._h, int(g), int(j), self.nrhs, ctypes.byref(self._p)),
              "hodlr_part_create")
        r0, nr, yc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(load().hodlr_part_info(self._p, ctypes.byref(r0), ctypes.byref(nr), ctypes.byref(yc)),
              "hodlr_part_info")
        self.row0, self.rows, self.yred_count = r0.value, nr.value, yc.value

    def _x(self, X: torch.Tensor) -> torch.Tensor:
        if (X.dim() != 2 or X.stride(1) != 1 or X.shape != (self.rows, self.nrhs) or X.dtype != self._m.dtype
                or not X.is_cuda):
            raise ValueError("X must be the part's (rows, nrhs) CUDA tensor of the working dtype, unit column stride")
        return X

    def new_yred(self) -> torch.Tensor:
        return torch.empty(max(self.yred_count, 1), dtype=self._m.dtype, device="cuda")

    def partial(self, X: torch.Tensor, yred: torch.Tensor, stream=None) -> None:
        X = self._x(X)
        if yred.numel() < self.yred_count or yred.dtype != self._m.dtype or not yred.is_contiguous():
            raise ValueError("yred must hold yred_count contiguous values of the working dtype")
        check(load().hodlr_part_partial(self._p, X.data_ptr(), X.stride(0), yred.data_ptr(), _stream_ptr(stream)),
              "hodlr_part_partial")

    def finish(self, X: torch.Tensor, yred: torch.Tensor, B: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        X = self._x(X)
        if B is None:
            B = torch.empty_like(X)
        if B.shape != X.shape or B.stride(1) != 1 or B.dtype != X.dtype or not B.is_cuda:
            raise ValueError("B must be a (rows, nrhs) CUDA tensor like X")
        if yred.numel() < self.yred_count or yred.dtype != self._m.dtype or not yred.is_contiguous():
            raise ValueError("yred must hold yred_count contiguous values of the working dtype")
        check(load().hodlr_part_finish(self._p, X.data_ptr(), X.stride(0), yred.data_ptr(), B.data_ptr(),
                                       B.stride(0), _stream_ptr(stream)), "hodlr_part_finish")
        return B

    def close(self):
        if self._p:
            load().hodlr_part_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tree_order(points, depth: int) -> np.ndarray:
    """hodlr_tree_order: the kd-tree order of ``points`` ((n, dim) or (n,)
    host array) for a cluster tree of the given depth; returns perm (int32)
    with points[perm] in tree order."""
    P = np.ascontiguousarray(np.asarray(points, dtype=np.float64))
    n = P.shape[0]
    P = P.reshape(n, -1)
    perm = np.empty(n, dtype=np.int32)
    check(load().hodlr_tree_order(n, P.shape[1], P.ctypes.data, int(depth),
                                  perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "hodlr_tree_order")
    return perm


def dense_kernel_matvec(points: torch.Tensor, kind: int, X: torch.Tensor, c: float = 0.0,
                        len2: float = 1.0, diag: float = 0.0, rows: torch.Tensor | None = None,
                        stream=None) -> torch.Tensor:
    """On-the-fly FP64 dense kernel product (hodlr_dense_kernel_matvec).
    points: (n, dim) fp64 CUDA; X: (n, R) fp64 CUDA; rows: int32 CUDA or None."""
    pts = points if points.dim() == 2 else points.view(-1, 1)
    pts = pts.contiguous()
    X2 = X.view(-1, 1) if X.dim() == 1 else X
    X2 = X2.contiguous()
    n, dim = pts.shape
    nrows = n if rows is None else rows.numel()
    B = torch.empty((nrows, X2.shape[1]), dtype=torch.float64, device=X2.device)
    rp = ctypes.c_void_p(rows.data_ptr()) if rows is not None else ctypes.c_void_p()
    check(load().hodlr_dense_kernel_matvec(n, dim, ctypes.c_void_p(pts.data_ptr()), kind, c, len2,
                                           diag, nrows, rp, X2.shape[1],
                                           ctypes.c_void_p(X2.data_ptr()), X2.shape[1],
                                           ctypes.c_void_p(B.data_ptr()), X2.shape[1],
                                           _stream_ptr(stream)), "hodlr_dense_kernel_matvec")
    return B
