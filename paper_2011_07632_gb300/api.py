"""Python binding of the spdhss C ABI (include/spdhss.h).

Thin argument marshalling over the CUDA library: PyTorch tensors supply device memory
and the current CUDA stream; every step of the method runs in the library's kernels.
Block vectors are (n, ncol) tensors in the original point order; they are handed to the
library column-major (a contiguous (ncol, n) buffer, leading dimension n).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import native as N


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _colmajor(X, device="cuda") -> torch.Tensor:
    """(n,) or (n, ncol) -> contiguous float64 (ncol, n) buffer on the device."""
    if isinstance(X, np.ndarray):
        X = torch.from_numpy(X)
    if X.dim() == 1:
        X = X[:, None]
    return X.to(device=device, dtype=torch.float64).t().contiguous()


def _i64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


class H2:
    """H^2 representation of sigma*I + K(X, X) (h2_build)."""

    def __init__(self, points, kernel: str = "exp", ell: float = 1.0, shift: float = 0.0,
                 leaf_size: int = 64, tol: float = 1e-8, stream=None):
        if isinstance(points, np.ndarray):
            points = torch.from_numpy(np.ascontiguousarray(points, dtype=np.float64))
        points = points.to(torch.float64).contiguous()
        n, dim = points.shape
        # matrix size: three unknowns per point for the RPY tensor kernel
        self.npoints, self.dim = int(n), int(dim)
        self.n = self.npoints * N.DOFS.get(kernel, 1)
        self.kernel, self.ell, self.shift = kernel, float(ell), float(shift)
        self.leaf_size, self.tol = int(leaf_size), float(tol)
        kd = N.KernelDesc(N.KERNELS[kernel], float(ell), float(shift))
        h = ctypes.c_void_p()
        N.check(N.lib().h2_build(_ptr(points), self.npoints, self.dim, kd, int(leaf_size), float(tol),
                                 _stream(stream), ctypes.byref(h)))
        self._h = h

    def matmul(self, X, stream=None) -> torch.Tensor:
        Xc = _colmajor(X)
        Yc = torch.empty_like(Xc)
        N.check(N.lib().h2_matmul(self._h, _ptr(Xc), _ptr(Yc), Xc.shape[0], self.n, _stream(stream)))
        return Yc.t()

    def matmul_mixed(self, X, stream=None) -> torch.Tensor:
        """Y = A X with the FP32 copy of the H^2 matrix (h2_matmul_mixed); at most 16 columns."""
        Xc = _colmajor(X)
        Yc = torch.empty_like(Xc)
        N.check(N.lib().h2_matmul_mixed(self._h, _ptr(Xc), _ptr(Yc), Xc.shape[0], self.n,
                                        _stream(stream)))
        return Yc.t()

    def info(self) -> dict:
        a = np.zeros(16, np.int64)
        N.check(N.lib().h2_info(self._h, _i64(a)))
        keys = ["n", "dim", "nodes", "D", "near_entries", "far_entries", "skeleton_total",
                "stored_bytes", "near_kernel_entries", "coupling_entries", "basis_entries",
                "max_rank"]
        return {k: int(a[i]) for i, k in enumerate(keys)}

    def export_tree(self) -> dict:
        inf = self.info()
        nn, D, dim = inf["nodes"], inf["D"], inf["dim"]
        out = {
            "perm": np.zeros(self.n, np.int64), "depth_off": np.zeros(D + 2, np.int64),
            "begin": np.zeros(nn, np.int64), "end": np.zeros(nn, np.int64),
            "parent": np.zeros(nn, np.int64), "cell_lo": np.zeros(nn * dim, np.int64),
            "cell_hi": np.zeros(nn * dim, np.int64), "near_off": np.zeros(nn + 1, np.int64),
            "near_idx": np.zeros(max(inf["near_entries"], 1), np.int64),
            "far_off": np.zeros(nn + 1, np.int64),
            "far_idx": np.zeros(max(inf["far_entries"], 1), np.int64),
        }
        order = ["perm", "depth_off", "begin", "end", "parent", "cell_lo", "cell_hi",
                 "near_off", "near_idx", "far_off", "far_idx"]
        N.check(N.lib().h2_export_tree(self._h, *[_i64(out[k]) for k in order]))
        out["near_idx"] = out["near_idx"][:inf["near_entries"]]
        out["far_idx"] = out["far_idx"][:inf["far_entries"]]
        out["cell_lo"] = out["cell_lo"].reshape(nn, dim)
        out["cell_hi"] = out["cell_hi"].reshape(nn, dim)
        out["D"] = D
        return out

    def export_skeletons(self):
        inf = self.info()
        off = np.zeros(inf["nodes"] + 1, np.int64)
        idx = np.zeros(max(inf["skeleton_total"], 1), np.int64)
        N.check(N.lib().h2_export_skeletons(self._h, _i64(off), _i64(idx)))
        return off, idx[:inf["skeleton_total"]]

    def close(self):
        if getattr(self, "_h", None):
            N.lib().h2_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HSS:
    """SPD HSS approximation built from an H^2 matrix (spdhss_build, Alg. 5.3)."""

    def __init__(self, h2: H2, rank: int, oversample: int = 10, omega=None, seed: int = 0,
                 stream=None, tol: float = 0.0, precision: int = 0):
        """tol > 0: bases truncated at that relative tolerance, rank being the cap
        (spdhss_build_tol).  precision 1 / 2: the sampling product in FP32 on the tensor
        cores, 3xTF32 / TF32 (spdhss_build_precision)."""
        self.h2 = h2
        self.rank, self.oversample, self.tol = int(rank), int(oversample), float(tol)
        om = None
        if omega is not None:
            om = _colmajor(omega)
            assert om.shape == (rank + oversample, h2.n)
        h = ctypes.c_void_p()
        N.check(N.lib().spdhss_build_precision(h2._h, int(rank), float(tol), int(oversample),
                                               _ptr(om) if om is not None else None, int(seed),
                                               int(precision), _stream(stream),
                                               ctypes.byref(h)))
        self._h = h

    def matmul(self, X, stream=None) -> torch.Tensor:
        Xc = _colmajor(X)
        Yc = torch.empty_like(Xc)
        N.check(N.lib().hss_matmul(self._h, _ptr(Xc), _ptr(Yc), Xc.shape[0], self.h2.n,
                                   _stream(stream)))
        return Yc.t()

    def info(self) -> dict:
        a = np.zeros(8, np.int64)
        N.check(N.lib().hss_info(self._h, _i64(a)))
        return {"levels": int(a[0]), "max_rank": int(a[1]), "stored_bytes": int(a[2]),
                "nodes": int(a[3])}

    def close(self):
        if getattr(self, "_h", None):
            N.lib().hss_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ULV:
    """ULV factorization of an SPD HSS matrix (ulv_factor / ulv_solve)."""

    def __init__(self, hss: HSS, stream=None):
        self.hss = hss
        h = ctypes.c_void_p()
        N.check(N.lib().ulv_factor(hss._h, _stream(stream), ctypes.byref(h)))
        self._h = h

    def solve(self, B, stream=None) -> torch.Tensor:
        Bc = _colmajor(B)
        Xc = torch.empty_like(Bc)
        N.check(N.lib().ulv_solve(self._h, _ptr(Bc), _ptr(Xc), Bc.shape[0], self.hss.h2.n,
                                  _stream(stream)))
        return Xc.t()

    def solve_noalloc(self, B, stream=None) -> torch.Tensor:
        """Same as solve(), through the entry point that allocates no device memory inside
        the library (fixed device arrays; see ulv_solve_noalloc in include/spdhss.h)."""
        Bc = _colmajor(B)
        Xc = torch.empty_like(Bc)
        N.check(N.lib().ulv_solve_noalloc(self._h, _ptr(Bc), _ptr(Xc), Bc.shape[0], self.hss.h2.n,
                                          _stream(stream)))
        return Xc.t()

    def close(self):
        if getattr(self, "_h", None):
            N.lib().ulv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_eval(kernel: str, ell: float, r2, stream=None) -> torch.Tensor:
    """K(r) at squared distances r2 (FP64, any shape), evaluated on the device the way the
    H^2 and SPD-HSS kernels evaluate it (scalar kernels only, no shift)."""
    r2 = torch.as_tensor(r2, dtype=torch.float64).cuda().contiguous()
    out = torch.empty_like(r2)
    N.check(N.lib().spdhss_kernel_eval(N.KernelDesc(N.KERNELS[kernel], float(ell), 0.0),
                                       _ptr(r2), _ptr(out), r2.numel(), _stream(stream)))
    return out


def pcg_solve(h2: H2, ulv: ULV, B, tol: float = 1e-6, maxit: int = 3000, stream=None,
              raise_on_no_convergence: bool = False, mixed: bool = False):
    """PCG (Sec. 6.2): returns (X (n, nrhs), iterations per column, true relres per column).
    mixed=True uses the FP32 product with A inside the iteration (pcg_solve_mixed);
    ulv=None runs unpreconditioned CG.

    B may be a CUDA tensor (device path) or a CPU tensor / numpy array (host buffers: the
    library stages them through the device and X comes back on the host)."""
    host = isinstance(B, np.ndarray) or (isinstance(B, torch.Tensor) and not B.is_cuda)
    Bc = _colmajor(B, device="cpu" if host else "cuda")
    if host:
        Bc = Bc.contiguous()
    nrhs = Bc.shape[0]
    Xc = torch.empty_like(Bc)
    it = (ctypes.c_int * nrhs)()
    rr = (ctypes.c_double * nrhs)()
    fn = N.lib().pcg_solve_mixed if mixed else N.lib().pcg_solve
    st = fn(h2._h, ulv._h if ulv is not None else None, _ptr(Bc), _ptr(Xc), nrhs, h2.n,
            float(tol), int(maxit), it, rr,
            _stream(stream))
    if st != N.OK and not (st == N.NO_CONVERGENCE and not raise_on_no_convergence):
        N.check(st)
    return Xc.t(), np.array(list(it)), np.array(list(rr))


def _wrap(cls, handle, **attrs):
    """A Python handle object around a library handle made by a batched call."""
    o = cls.__new__(cls)
    for k, v in attrs.items():
        setattr(o, k, v)
    o._h = ctypes.c_void_p(handle) if handle else None
    return o


def build_batched(instances, stream=None):
    """Batched level sweep (spdhss_build_batched): H^2 -> SPD-HSS -> ULV for independent
    instances, with the batched kernel launches of all instances merged step by step.

    instances: list of dicts with keys points ((n, dim) array or tensor), kernel, ell,
    shift, leaf_size, tol, rank, oversample (default 10), seed (default 0), omega (optional
    (n, rank + oversample) sketch, else drawn on the device from seed), precision (0 FP64,
    1 / 2 the sampling product on the tensor cores, as HSS(precision=...)).
    Returns (list of (H2, HSS, ULV) or None per instance, per-instance status codes,
    (merged launches, hand-overs))."""
    m = len(instances)
    pts, keep = [], []
    for inst in instances:
        p = inst["points"]
        if isinstance(p, np.ndarray):
            p = torch.from_numpy(np.ascontiguousarray(p, dtype=np.float64))
        p = p.to(torch.float64).contiguous()
        keep.append(p)
        pts.append(p)
    ptr = (ctypes.c_void_p * m)(*[p.data_ptr() for p in pts])
    n = np.array([p.shape[0] for p in pts], np.int64)
    dim = (ctypes.c_int * m)(*[int(p.shape[1]) for p in pts])
    kd = (N.KernelDesc * m)(*[N.KernelDesc(N.KERNELS[i["kernel"]], float(i["ell"]),
                                            float(i["shift"])) for i in instances])
    leaf = (ctypes.c_int * m)(*[int(i["leaf_size"]) for i in instances])
    tol = (ctypes.c_double * m)(*[float(i["tol"]) for i in instances])
    rank = (ctypes.c_int * m)(*[int(i["rank"]) for i in instances])
    over = (ctypes.c_int * m)(*[int(i.get("oversample", 10)) for i in instances])
    seed = (ctypes.c_uint64 * m)(*[int(i.get("seed", 0)) for i in instances])
    oms = []
    for k, inst in enumerate(instances):
        om = inst.get("omega")
        if om is not None:
            om = _colmajor(om)
            assert om.shape == (int(inst["rank"]) + int(inst.get("oversample", 10)),
                                int(pts[k].shape[0]))
        oms.append(om)
    keep.extend(o for o in oms if o is not None)
    omp = (ctypes.c_void_p * m)(*[o.data_ptr() if o is not None else None for o in oms])
    prec = (ctypes.c_int * m)(*[int(i.get("precision", 0)) for i in instances])
    h2o, hso, ulo = (ctypes.c_void_p * m)(), (ctypes.c_void_p * m)(), (ctypes.c_void_p * m)()
    st = (ctypes.c_int * m)()
    rc = N.lib().spdhss_build_batched(m, ptr, _i64(n), dim, kd, leaf, tol, rank, over, seed,
                                      omp, prec, _stream(stream), h2o, hso, ulo, st)
    if rc != N.OK and all(v == N.OK for v in st):
        N.check(rc)
    out = []
    for k, inst in enumerate(instances):
        if st[k] != N.OK:
            out.append(None)
            continue
        h = _wrap(H2, h2o[k], n=int(n[k]) * N.DOFS.get(inst["kernel"], 1), npoints=int(n[k]),
                  dim=int(dim[k]), kernel=inst["kernel"],
                  ell=float(inst["ell"]), shift=float(inst["shift"]),
                  leaf_size=int(inst["leaf_size"]), tol=float(inst["tol"]))
        hs = _wrap(HSS, hso[k], h2=h, rank=int(inst["rank"]),
                   oversample=int(inst.get("oversample", 10)))
        u = _wrap(ULV, ulo[k], hss=hs)
        out.append((h, hs, u))
    stats = np.zeros(2, np.int64)
    N.lib().spdhss_batched_stats(_i64(stats))
    return out, [int(v) for v in st], (int(stats[0]), int(stats[1]))


def pcg_solve_batched(h2s, ulvs, Bs, tol: float = 1e-6, maxit: int = 3000, stream=None,
                      mixed: bool = False, on_done=None):
    """pcg_solve for every instance with the iterations in lockstep (pcg_solve_batched;
    mixed=True: pcg_solve_mixed per instance, pcg_solve_batched_mixed, at most 16 columns).
    Bs: device tensors or arrays (n_i, nrhs_i).  Returns (list of X (n_i, nrhs_i) device
    tensors, list of iteration arrays, list of relres arrays, per-instance status codes).
    on_done(i, status, X_i, iters_i, relres_i), if given, is called as soon as instance i
    has finished (pcg_solve_batched_ex), with its final results; it must not destroy the
    instances' handles."""
    m = len(h2s)
    Bc = [_colmajor(b) for b in Bs]
    Xc = [torch.empty_like(b) for b in Bc]
    nrhs = [b.shape[0] for b in Bc]
    its = [(ctypes.c_int * k)() for k in nrhs]
    rrs = [(ctypes.c_double * k)() for k in nrhs]
    P = ctypes.c_void_p * m
    ld = np.array([h.n for h in h2s], np.int64)
    st = (ctypes.c_int * m)()
    args = (m, P(*[h._h.value for h in h2s]), P(*[u._h.value for u in ulvs]),
            P(*[b.data_ptr() for b in Bc]), P(*[x.data_ptr() for x in Xc]),
            (ctypes.c_int * m)(*nrhs), _i64(ld), float(tol), int(maxit),
            P(*[ctypes.addressof(a) for a in its]), P(*[ctypes.addressof(a) for a in rrs]),
            _stream(stream), st)
    if on_done is not None:
        def _done(_user, k, status):
            on_done(k, int(status), Xc[k].t(), np.array(list(its[k])), np.array(list(rrs[k])))
        cb = N.DONE_FN(_done)   # referenced until the call returns
        rc = N.lib().pcg_solve_batched_ex(*args, 1 if mixed else 0, cb, None)
    else:
        fn = N.lib().pcg_solve_batched_mixed if mixed else N.lib().pcg_solve_batched
        rc = fn(*args)
    if any(v not in (N.OK, N.NO_CONVERGENCE) for v in st) or (
            rc != N.OK and all(v == N.OK for v in st)):
        N.check(rc)
    return ([x.t() for x in Xc], [np.array(list(a)) for a in its],
            [np.array(list(a)) for a in rrs], [int(v) for v in st])
