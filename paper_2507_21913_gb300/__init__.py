"""Python binding of the hpfmm C ABI (``include/hpfmm.h``): argument
marshalling only.  Every step of the evaluation runs in the CUDA library
``_lib/libhpfmm.so`` (built by ``_build.build()``); there is no CPU fallback,
and importing the functions without the built library raises.

Inputs may be torch tensors (CUDA or CPU) or numpy arrays; CPU inputs go
through the library's host-pointer path (stream-ordered staging copies).
Outputs are complex128 torch tensors on the device of the inputs.
"""
import ctypes
import os

import numpy as np

from . import _build

HPFMM_OK, HPFMM_EINVAL, HPFMM_ENOMEM, HPFMM_ECUDA, HPFMM_ETIMEOUT, HPFMM_EUNSUPPORTED = range(6)
PRECISIONS = {"fp64": 0, "fp32": 1, "mixed": 2}

_LIB = None


class HpfmmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("hpfmm status %d (%s): %s" % (status, _LIB.hpfmm_status_string(status).decode()
                                                        if _LIB else "?", msg))
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("tau_fp64", ctypes.c_double), ("levels", ctypes.c_int),
                ("subtree_levels", ctypes.c_int), ("m2l_mode", ctypes.c_int),
                ("adaptive", ctypes.c_int), ("async_update", ctypes.c_int),
                ("reserved", ctypes.c_int * 1),
                ("root_x0", ctypes.c_double),
                ("root_side", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("levels", ctypes.c_int), ("subtree_levels", ctypes.c_int),
                ("met", ctypes.c_int), ("mean_leaf", ctypes.c_double),
                ("est_rel_err", ctypes.c_double), ("ms_per_eval", ctypes.c_double),
                ("nsample", ctypes.c_int)]


class AluPeaks(ctypes.Structure):
    _fields_ = [("sms", ctypes.c_int), ("mufu_ops_per_s", ctypes.c_double),
                ("ffma_flops_per_s", ctypes.c_double), ("dfma_flops_per_s", ctypes.c_double),
                ("mufu_mhz", ctypes.c_double), ("ffma_mhz", ctypes.c_double),
                ("dfma_mhz", ctypes.c_double), ("mufu_per_clk_sm", ctypes.c_double),
                ("ffma_flops_per_clk_sm", ctypes.c_double),
                ("dfma_flops_per_clk_sm", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("levels", ctypes.c_int), ("p", ctypes.c_int),
                ("prec", ctypes.c_int), ("x0", ctypes.c_double), ("side", ctypes.c_double),
                ("workspace_bytes", ctypes.c_int64)]


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False):
    """Load the CUDA library.  Raises if it has not been built (no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError("hpfmm CUDA library not built (%s); run "
                               "__graft_entry__.build() or paper_2507_21913_gb300._build.build()"
                               % path)
    L = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.hpfmm_create.argtypes = [vp, vp, i64, dbl, dbl, i32, i32, ctypes.POINTER(Options), vp,
                               ctypes.POINTER(vp)]
    L.hpfmm_eval.argtypes = [vp, vp, i32, vp, vp, vp]
    L.hpfmm_update_points.argtypes = [vp, vp, vp, vp]
    L.hpfmm_destroy.argtypes = [vp]
    L.hpfmm_direct.argtypes = [vp, vp, vp, i64, vp, vp, vp, i64, dbl, dbl, vp, vp, vp]
    L.hpfmm_get_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    L.hpfmm_get_order.argtypes = [vp, vp, vp, vp]
    L.hpfmm_sync.argtypes = [vp, vp]
    L.hpfmm_set_timing.argtypes = [vp, i32]
    L.hpfmm_selftest_wait_timeout.argtypes = [vp]
    L.hpfmm_tree_order_noalloc.argtypes = [vp, vp, i64, i32, vp, vp, vp]
    L.hpfmm_read_timing.argtypes = [vp, vp, vp]
    L.hpfmm_read_timeline.argtypes = [vp, i32, vp, vp, vp, ctypes.POINTER(i32)]
    L.hpfmm_eval_adjoint.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.hpfmm_batch_create.argtypes = [vp, i32, i32, ctypes.POINTER(vp)]
    L.hpfmm_eval_batched.argtypes = [vp, vp, vp, vp, vp]
    L.hpfmm_batch_captures.argtypes = [vp, ctypes.POINTER(i64)]
    L.hpfmm_batch_destroy.argtypes = [vp]
    L.hpfmm_autotune.argtypes = [vp, vp, i64, dbl, dbl, i32, dbl, i32, vp, ctypes.POINTER(Tuning)]
    L.hpfmm_selftest_tc_gemm.argtypes = [vp, vp, vp, i32, i32, i32, vp]
    L.hpfmm_eval_targets.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp]
    L.hpfmm_get_adaptive_counts.argtypes = [vp, i32, vp, vp, vp, vp]
    L.hpfmm_measure_alu_peaks.argtypes = [ctypes.POINTER(AluPeaks), vp]
    L.hpfmm_default_options.argtypes = [ctypes.POINTER(Options)]
    L.hpfmm_default_options.restype = None
    for f in ("hpfmm_create", "hpfmm_eval", "hpfmm_update_points", "hpfmm_destroy", "hpfmm_direct", "hpfmm_get_info",
              "hpfmm_get_order", "hpfmm_sync", "hpfmm_set_timing", "hpfmm_read_timing",
              "hpfmm_selftest_wait_timeout", "hpfmm_tree_order_noalloc", "hpfmm_eval_adjoint",
              "hpfmm_batch_create", "hpfmm_eval_batched", "hpfmm_batch_captures",
              "hpfmm_batch_destroy", "hpfmm_autotune", "hpfmm_selftest_tc_gemm",
              "hpfmm_eval_targets", "hpfmm_get_adaptive_counts", "hpfmm_measure_alu_peaks"):
        getattr(L, f).restype = ctypes.c_int
    L.hpfmm_status_string.argtypes = [ctypes.c_int]
    L.hpfmm_status_string.restype = ctypes.c_char_p
    L.hpfmm_last_error.restype = ctypes.c_char_p
    L.hpfmm_version.restype = ctypes.c_char_p
    _LIB = L
    return L


def _check(status):
    if status != HPFMM_OK:
        raise HpfmmError(status, lib().hpfmm_last_error().decode())


def _torch():
    import torch
    return torch


def _as_tensor(a, device=None):
    torch = _torch()
    if isinstance(a, np.ndarray) or not hasattr(a, "data_ptr"):
        a = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64))
    if a.dtype != torch.float64:
        a = a.to(torch.float64)
    if device is not None and a.device != device:
        a = a.to(device)
    return a.contiguous()


def _stream(device):
    torch = _torch()
    if device.type == "cuda":
        return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    return ctypes.c_void_p(0)


class Plan:
    """An hpfmm plan (tree, tables and workspace for one point set)."""

    def __init__(self, handle, n, device):
        self.handle = handle
        self.n = n
        self.device = device

    def info(self):
        return hpfmm_get_info(self)

    def __del__(self):
        try:
            if self.handle:
                lib().hpfmm_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def hpfmm_create(x, y, kappa=1.0, p=12, leaf_size=32, prec="fp64", levels=0, tau_fp64=0.05,
                 subtree_levels=0, m2l_mode=0, root=None, adaptive=False, async_update=False):
    """Build a plan for the points (x, y); see hpfmm_create in include/hpfmm.h."""
    x = _as_tensor(x)
    y = _as_tensor(y, x.device)
    kappa = complex(kappa)
    opt = Options()
    lib().hpfmm_default_options(ctypes.byref(opt))
    opt.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    opt.levels = int(levels)
    opt.tau_fp64 = float(tau_fp64)
    opt.subtree_levels = int(subtree_levels)
    opt.m2l_mode = int(m2l_mode)
    opt.adaptive = 1 if adaptive else 0
    opt.async_update = 1 if async_update else 0
    if root is not None:  # (x0, side): the tree's root square
        opt.root_x0, opt.root_side = float(root[0]), float(root[1])
    h = ctypes.c_void_p()
    _check(lib().hpfmm_create(x.data_ptr(), y.data_ptr(), x.numel(), kappa.real, kappa.imag,
                              int(p), int(leaf_size), ctypes.byref(opt), _stream(x.device),
                              ctypes.byref(h)))
    return Plan(h, x.numel(), x.device)


def hpfmm_update_points(plan, x, y):
    """Rebuild the plan's tree and tables for new points (same n), no allocation."""
    x = _as_tensor(x)
    y = _as_tensor(y, x.device)
    if x.numel() != plan.n or y.numel() != plan.n:
        raise ValueError("hpfmm_update_points: expected %d points" % plan.n)
    _check(lib().hpfmm_update_points(plan.handle, x.data_ptr(), y.data_ptr(), _stream(x.device)))


def hpfmm_eval(plan, q, grad=True, out=None):
    """u = G q (and grad u) for q of shape (n,) or (nrhs, n).  Returns complex128
    tensors pot (nrhs, n) and grad (nrhs, n, 2) (or None), squeezed for 1-D q.
    out=(pot, grad) supplies the output tensors (e.g. pinned host memory)."""
    torch = _torch()
    q = _as_tensor(q)
    squeeze = q.dim() == 1
    q2 = q.reshape(-1, plan.n)
    nrhs = q2.shape[0]
    if out is not None:
        pot, g = out
        pot = pot.view(nrhs, plan.n)
        g = g.view(nrhs, plan.n, 2) if (grad and g is not None) else None
        grad = g is not None
    else:
        pot = torch.empty((nrhs, plan.n), dtype=torch.complex128, device=q.device)
        g = torch.empty((nrhs, plan.n, 2), dtype=torch.complex128, device=q.device) if grad else None
    _check(lib().hpfmm_eval(plan.handle, q2.data_ptr(), nrhs, pot.data_ptr(),
                            g.data_ptr() if grad else None, _stream(q.device)))
    if squeeze:
        return pot[0], (g[0] if grad else None)
    return pot, g


def hpfmm_eval_adjoint(plan, q, g, grad_q=None, want_q=True, want_r=True):
    """Gradient of a real functional L of u = G q (see hpfmm_eval_adjoint in
    include/hpfmm.h): g = dL/dRe u + i dL/dIm u (complex, shape (n,)).
    Returns (dq (n,) or None, dxy (n, 2) or None) as float64 device tensors."""
    torch = _torch()
    dev = plan.device
    if dev.type != "cuda":
        raise ValueError("hpfmm_eval_adjoint needs device tensors")
    g = torch.as_tensor(g, device=dev).to(torch.complex128).contiguous().reshape(plan.n)
    q = _as_tensor(q, dev).reshape(plan.n) if q is not None else None
    if grad_q is not None:
        grad_q = torch.as_tensor(grad_q, device=dev).to(torch.complex128).contiguous()
    dq = torch.empty(plan.n, dtype=torch.float64, device=dev) if want_q else None
    dxy = torch.empty((plan.n, 2), dtype=torch.float64, device=dev) if want_r else None
    _check(lib().hpfmm_eval_adjoint(plan.handle, q.data_ptr() if q is not None else None,
                                    g.data_ptr(), grad_q.data_ptr() if grad_q is not None else None,
                                    dq.data_ptr() if dq is not None else None,
                                    dxy.data_ptr() if dxy is not None else None, _stream(dev)))
    return dq, dxy


def _autograd_function():
    torch = _torch()

    class HalfPlanePotential(torch.autograd.Function):
        """u = G q on the plan's points; backward by hpfmm_eval_adjoint."""

        @staticmethod
        def forward(ctx, x, y, q, plan):
            want_r = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
            pot, gq = hpfmm_eval(plan, q.detach(), grad=want_r)
            ctx.plan = plan
            ctx.save_for_backward(q.detach(), gq if want_r else None)
            return pot

        @staticmethod
        def backward(ctx, g):
            q, gq = ctx.saved_tensors
            want_r = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
            dq, dxy = hpfmm_eval_adjoint(ctx.plan, q, g, grad_q=gq,
                                         want_q=ctx.needs_input_grad[2], want_r=want_r)
            dx = dxy[:, 0] if (want_r and ctx.needs_input_grad[0]) else None
            dy = dxy[:, 1] if (want_r and ctx.needs_input_grad[1]) else None
            return dx, dy, dq, None

    return HalfPlanePotential


_HPP = None


def potential(x, y, q, kappa=1.0, p=12, leaf_size=32, prec="fp64", levels=0, plan=None):
    """Differentiable u = G q (complex128, shape (n,)) for float64 device tensors
    x, y, q.  The plan (tree, tables) is built on x, y, or, when given, rebuilt
    in place for them; gradients with respect to x, y and q come from
    hpfmm_eval_adjoint."""
    global _HPP
    if _HPP is None:
        _HPP = _autograd_function()
    if plan is None:
        plan = hpfmm_create(x.detach(), y.detach(), kappa=kappa, p=p, leaf_size=leaf_size,
                            prec=prec, levels=levels)
    else:
        hpfmm_update_points(plan, x.detach(), y.detach())
    return _HPP.apply(x, y, q, plan)


class Batch:
    """Independent problems evaluated as one CUDA graph (hpfmm_batch_* in
    include/hpfmm.h).  Holds references to its plans and its output tensors,
    which stay the same between calls so that the graph is replayed."""

    def __init__(self, handle, plans):
        self.handle = handle
        self.plans = list(plans)
        self.out = {}

    def captures(self):
        c = ctypes.c_int64()
        _check(lib().hpfmm_batch_captures(self.handle, ctypes.byref(c)))
        return c.value

    def __del__(self):
        try:
            if self.handle:
                lib().hpfmm_batch_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def hpfmm_batch_create(plans, nbranch=0):
    arr = (ctypes.c_void_p * len(plans))(*[p.handle.value if isinstance(p.handle, ctypes.c_void_p)
                                            else p.handle for p in plans])
    h = ctypes.c_void_p()
    _check(lib().hpfmm_batch_create(arr, len(plans), int(nbranch), ctypes.byref(h)))
    return Batch(h, plans)


def hpfmm_eval_batched(batch, qs, grad=True):
    """Evaluate every problem of the batch (qs[i]: float64 device tensor of the
    plan's n).  Returns lists (pot[i], grad[i] or None); the tensors belong to
    the batch and are overwritten by its next call with the same grad flag."""
    torch = _torch()
    plans = batch.plans
    if len(qs) != len(plans):
        raise ValueError("hpfmm_eval_batched: %d charge vectors for %d plans" % (len(qs), len(plans)))
    qs = [_as_tensor(q, p.device).reshape(p.n) for q, p in zip(qs, plans)]
    key = bool(grad)
    if key not in batch.out:
        batch.out[key] = (
            [torch.empty(p.n, dtype=torch.complex128, device=p.device) for p in plans],
            [torch.empty((p.n, 2), dtype=torch.complex128, device=p.device) for p in plans]
            if grad else None)
    pots, grads = batch.out[key]
    vp = ctypes.c_void_p
    qa = (vp * len(plans))(*[q.data_ptr() for q in qs])
    pa = (vp * len(plans))(*[t.data_ptr() for t in pots])
    ga = (vp * len(plans))(*[t.data_ptr() for t in grads]) if grad else None
    batch._keep = qs  # the graph reads these until the call has run
    _check(lib().hpfmm_eval_batched(batch.handle, qa, pa, ga, _stream(plans[0].device)))
    return pots, grads


def hpfmm_autotune(x, y, kappa=1.0, prec="fp32", tol=1e-6, nsample=256):
    """Pick p, levels and subtree_levels by measurement (see include/hpfmm.h).
    Returns a dict; pass p, levels and subtree_levels on to hpfmm_create."""
    x = _as_tensor(x)
    y = _as_tensor(y, x.device)
    kappa = complex(kappa)
    t = Tuning()
    _check(lib().hpfmm_autotune(x.data_ptr(), y.data_ptr(), x.numel(), kappa.real, kappa.imag,
                                PRECISIONS[prec] if isinstance(prec, str) else int(prec),
                                float(tol), int(nsample), _stream(x.device), ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in Tuning._fields_}


def hpfmm_eval_targets(plan, q, xt, yt, grad=True):
    """u (and grad u) at separate targets (xt, yt) from the plan's sources with
    charges q; see include/hpfmm.h.  Device tensors; returns complex128
    (nt,) and (nt, 2) or None."""
    torch = _torch()
    dev = plan.device
    q = _as_tensor(q, dev).reshape(plan.n)
    xt = _as_tensor(xt, dev).reshape(-1)
    yt = _as_tensor(yt, dev).reshape(-1)
    nt = xt.numel()
    pot = torch.empty(nt, dtype=torch.complex128, device=dev)
    g = torch.empty((nt, 2), dtype=torch.complex128, device=dev) if grad else None
    _check(lib().hpfmm_eval_targets(plan.handle, q.data_ptr(), xt.data_ptr(), yt.data_ptr(), nt,
                                    pot.data_ptr(), g.data_ptr() if grad else None, _stream(dev)))
    return pot, g


def hpfmm_destroy(plan):
    if plan.handle:
        _check(lib().hpfmm_destroy(plan.handle))
        plan.handle = None


def hpfmm_direct(xs, ys, qs, xt=None, yt=None, kappa=1.0, self_index=None, grad=True):
    """All-pairs device evaluation (double precision).  With xt/yt omitted the
    targets are the sources and the free part skips j == i."""
    torch = _torch()
    xs = _as_tensor(xs)
    dev = xs.device
    ys = _as_tensor(ys, dev)
    qs = _as_tensor(qs, dev)
    if xt is None:
        xt, yt = xs, ys
        if self_index is None:
            self_index = torch.arange(xs.numel(), dtype=torch.int64, device=dev)
    else:
        xt = _as_tensor(xt, dev)
        yt = _as_tensor(yt, dev)
    si = None
    if self_index is not None:
        si = torch.as_tensor(self_index, dtype=torch.int64, device=dev).contiguous()
    nt = xt.numel()
    kappa = complex(kappa)
    pot = torch.empty(nt, dtype=torch.complex128, device=dev)
    g = torch.empty((nt, 2), dtype=torch.complex128, device=dev) if grad else None
    _check(lib().hpfmm_direct(xs.data_ptr(), ys.data_ptr(), qs.data_ptr(), xs.numel(),
                              xt.data_ptr(), yt.data_ptr(), si.data_ptr() if si is not None else None,
                              nt, kappa.real, kappa.imag, pot.data_ptr(),
                              g.data_ptr() if grad else None, _stream(dev)))
    return pot, g


def hpfmm_get_adaptive_counts(plan, maxlev=13):
    """(boxes[l], leaves[l]) for l = 0..maxlev and the depth of an adaptive plan's tree."""
    boxes = np.zeros(maxlev + 1, np.int64)
    leaves = np.zeros(maxlev + 1, np.int64)
    depth = ctypes.c_int()
    _check(lib().hpfmm_get_adaptive_counts(plan.handle, int(maxlev), boxes.ctypes.data,
                                           leaves.ctypes.data, ctypes.byref(depth),
                                           _stream(plan.device)))
    return boxes, leaves, depth.value


def hpfmm_get_info(plan):
    info = PlanInfo()
    _check(lib().hpfmm_get_info(plan.handle, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in PlanInfo._fields_}


def hpfmm_get_order(plan):
    """(keys uint64 numpy, perm int64 numpy) of the plan's tree order."""
    keys = np.zeros(plan.n, np.uint64)
    perm = np.zeros(plan.n, np.int64)
    _check(lib().hpfmm_get_order(plan.handle, keys.ctypes.data, perm.ctypes.data,
                                 _stream(plan.device)))
    return keys, perm


PASS_NAMES = ("tree", "tables", "gather", "p2m", "m2m", "m2l_free", "m2l_mirror", "l2l", "eval",
              "near_mirror")


def hpfmm_set_timing(plan, enable=True):
    _check(lib().hpfmm_set_timing(plan.handle, 1 if enable else 0))


def hpfmm_read_timing(plan):
    """({pass: device ms since the last read}, {pass: kernel launches since creation})."""
    ms = np.zeros(len(PASS_NAMES))
    ln = np.zeros(len(PASS_NAMES), np.int64)
    _check(lib().hpfmm_read_timing(plan.handle, ms.ctypes.data, ln.ctypes.data))
    return dict(zip(PASS_NAMES, ms.tolist())), dict(zip(PASS_NAMES, ln.tolist()))


def hpfmm_read_timeline(plan, cap=4096):
    """[(pass name, begin ms, end ms)] of the pass intervals recorded since the
    last read, offsets from the earliest begin (see include/hpfmm.h)."""
    ps = np.zeros(cap, np.int32)
    b = np.zeros(cap)
    e = np.zeros(cap)
    cnt = ctypes.c_int32(0)
    _check(lib().hpfmm_read_timeline(plan.handle, cap, ps.ctypes.data, b.ctypes.data,
                                     e.ctypes.data, ctypes.byref(cnt)))
    return [(PASS_NAMES[int(ps[i])], float(b[i]), float(e[i])) for i in range(cnt.value)]


def hpfmm_sync(plan):
    _check(lib().hpfmm_sync(plan.handle, _stream(plan.device)))


def hpfmm_selftest_wait_timeout(device=None):
    """Run the bounded-wait failure self-test; returns the status code
    (HPFMM_ETIMEOUT is the expected outcome)."""
    import torch
    dev = torch.device(device or "cuda:0")
    return int(lib().hpfmm_selftest_wait_timeout(_stream(dev)))


def hpfmm_tree_order_noalloc(x, y, levels=5):
    """Tree ordering (sorted keys, permutation) without device allocations by the
    library (n <= 65536, device tensors); see include/hpfmm.h."""
    import torch
    x = _as_tensor(x)
    dev = x.device if x.device.type == "cuda" else torch.device("cuda", torch.cuda.current_device())
    x = _as_tensor(x, dev)
    y = _as_tensor(y, dev)
    keys = torch.empty(x.numel(), dtype=torch.int64, device=dev)
    perm = torch.empty(x.numel(), dtype=torch.int64, device=dev)
    with torch.cuda.device(dev):
        _check(lib().hpfmm_tree_order_noalloc(x.data_ptr(), y.data_ptr(), x.numel(), int(levels),
                                              keys.data_ptr(), perm.data_ptr(), _stream(dev)))
    return keys.cpu().numpy().view(np.uint64), perm.cpu().numpy()


def hpfmm_selftest_tc_gemm(A, B, split=True):
    """D = A B^T on the tensor cores (tf32, or the three-term split); A: 128 x k,
    B: n x k float32 device tensors.  Returns D (128 x n float32)."""
    torch = _torch()
    A = A.to(torch.float32).contiguous()
    B = B.to(torch.float32).contiguous()
    D = torch.empty((A.shape[0], B.shape[0]), dtype=torch.float32, device=A.device)
    _check(lib().hpfmm_selftest_tc_gemm(A.data_ptr(), B.data_ptr(), D.data_ptr(), B.shape[0],
                                        A.shape[1], 1 if split else 0, _stream(A.device)))
    return D


def hpfmm_measure_alu_peaks(device=None):
    """Measured SFU / FP32 FMA / FP64 FMA throughput of the device (see
    include/hpfmm.h); returns a dict."""
    torch = _torch()
    dev = torch.device(device or "cuda:0")
    r = AluPeaks()
    with torch.cuda.device(dev):
        _check(lib().hpfmm_measure_alu_peaks(ctypes.byref(r), _stream(dev)))
    return {f: getattr(r, f) for f, _ in AluPeaks._fields_}


def hpfmm_version():
    return lib().hpfmm_version().decode()
