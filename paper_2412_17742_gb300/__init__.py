"""Python binding of the gbsbin C ABI (``include/gbsbin.h``).

Argument marshalling only: every step of the computation runs in the CUDA library
``lib/libgbsbin.so``; there is no CPU fallback.  If the library is missing, :func:`load`
raises.  Functions carry the names of the C entry points; PyTorch is used only for device
buffers and the current stream.

Binned photon-number distributions of Gaussian states by evaluating the generating
function q(A, gamma, D(w)) / q(A, gamma, 1) on a roots-of-unity grid and taking an
inverse DFT (arXiv:2412.17742, Sec. III Eq. q_d, Sec. VI Eqs. Lamb_lhaf_master and
coarse_grained_prob).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libgbsbin.so")
_lib = None

GBSBIN_FP64 = 0
GBSBIN_FP32_REFINE = 1
KERNELS = {1: "smem_fp64", 2: "smem_fp32r", 3: "gmem_fp64", 4: "gmem_fp32r", 5: "warp_fp32r", 6: "blk_fp32r",
           7: "blk_tc_fp32r", 8: "hess_fp64", 9: "fock_fp64", 10: "fock_df32",
           11: "tree_df32", 12: "tree_fp64", 13: "btree_df32", 14: "btree_fp64", 15: "herald_fp64",
           16: "hess_df32"}
EXPORTED = ["gbsbin_default_options", "gbsbin_plan_create", "gbsbin_plan_set_state", "gbsbin_plan_destroy",
            "gbsbin_plan_table_size", "gbsbin_execute", "gbsbin_execute_host", "gbsbin_execute_host_async",
            "gbsbin_diagnostics",
            "gbsbin_strerror", "gbsbin_alu_peak", "gbsbin_read_points", "gbsbin_table_from_logq_noalloc",
            "gbsbin_backward", "gbsbin_backward_device", "gbsbin_autotune", "gbsbin_batch_create", "gbsbin_batch_execute",
            "gbsbin_batch_capture_graph", "gbsbin_batch_replay", "gbsbin_batch_table_size",
            "gbsbin_batch_diagnostics", "gbsbin_batch_read_points", "gbsbin_batch_destroy", "gbsbin_moments",
            "gbsbin_fock_plan_create", "gbsbin_fock_plan_set_transfer", "gbsbin_fock_plan_table_size",
            "gbsbin_fock_execute", "gbsbin_fock_execute_host", "gbsbin_fock_diagnostics",
            "gbsbin_fock_plan_destroy", "gbsbin_cumulants3", "gbsbin_cumulants4", "gbsbin_fock_plan_nodes",
            "gbsbin_total_photon_series", "gbsbin_cumulant_groups", "gbsbin_prob_distinguishable",
            "gbsbin_prob_distinguishable_device", "gbsbin_cumulants_device", "gbsbin_herald_plan_create", "gbsbin_herald_table_size",
            "gbsbin_herald_prob_size", "gbsbin_herald_execute", "gbsbin_herald_execute_host",
            "gbsbin_herald_diagnostics", "gbsbin_herald_plan_destroy"]
GBSBIN_HERALD_TRACED = -1
GBSBIN_HERALD_KEPT = -2


class GbsbinError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: status {status} ({gbsbin_strerror(status)})")


class gbsbin_complex(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class gbsbin_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("oversample", ctypes.c_int),
                ("want_diagnostics", ctypes.c_int), ("tile_override", ctypes.c_int),
                ("want_timing", ctypes.c_int), ("want_backward", ctypes.c_int),
                ("shard_begin", ctypes.c_longlong), ("shard_end", ctypes.c_longlong)]


_cp = ctypes.POINTER(gbsbin_complex)
_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)


class gbsbin_problem(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("K", ctypes.c_int), ("r", _dp), ("T", _cp), ("alpha", _cp), ("V", _cp),
                ("sigma1", _cp), ("zbar", _cp), ("bin_of_mode", _ip), ("L", ctypes.c_int), ("cutoff", _ip)]


class gbsbin_grads(ctypes.Structure):
    _fields_ = [("d_r", _dp), ("d_T", _cp), ("d_alpha", _cp), ("d_V", _cp), ("d_sigma1", _cp), ("d_zbar", _cp)]


class gbsbin_diag(ctypes.Structure):
    _fields_ = [("sum_P", ctypes.c_double), ("max_imag", ctypes.c_double), ("min_pivot_re", ctypes.c_double),
                ("n_bad_points", ctypes.c_longlong), ("n_points", ctypes.c_longlong),
                ("n_evaluated", ctypes.c_longlong), ("table_size", ctypes.c_longlong), ("n", ctypes.c_int),
                ("kernel", ctypes.c_int), ("log_q1_re", ctypes.c_double), ("point_kernel_ms", ctypes.c_double),
                ("state_upload_bytes", ctypes.c_longlong), ("launches", ctypes.c_int),
                ("backward_kernel_ms", ctypes.c_double), ("backward_path", ctypes.c_int)]


class gbsbin_fock_problem(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("T", _cp), ("photons", _ip), ("bin_of_mode", _ip), ("L", ctypes.c_int),
                ("cutoff", _ip)]


class gbsbin_herald_problem(ctypes.Structure):
    _fields_ = [("state", gbsbin_problem), ("role", _ip), ("L", ctypes.c_int), ("cutoff", _ip),
                ("fock_cutoff", ctypes.c_int)]


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"gbsbin CUDA library not built: {LIB_PATH} is missing "
                           "(run paper_2412_17742_gb300/build.py)")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    lib.gbsbin_default_options.argtypes = [ctypes.POINTER(gbsbin_options)]
    lib.gbsbin_default_options.restype = None
    lib.gbsbin_plan_create.argtypes = [ctypes.POINTER(gbsbin_problem), ctypes.POINTER(gbsbin_options),
                                       ctypes.POINTER(vp)]
    lib.gbsbin_plan_set_state.argtypes = [vp, ctypes.POINTER(gbsbin_problem), vp]
    lib.gbsbin_plan_destroy.argtypes = [vp]
    lib.gbsbin_plan_table_size.argtypes = [vp]
    lib.gbsbin_plan_table_size.restype = ctypes.c_longlong
    lib.gbsbin_execute.argtypes = [vp, vp, vp]
    lib.gbsbin_execute_host.argtypes = [vp, vp, vp]
    lib.gbsbin_execute_host_async.argtypes = [vp, vp, vp]
    lib.gbsbin_diagnostics.argtypes = [vp, ctypes.POINTER(gbsbin_diag), vp]
    lib.gbsbin_strerror.argtypes = [ctypes.c_int]
    lib.gbsbin_strerror.restype = ctypes.c_char_p
    lib.gbsbin_alu_peak.argtypes = [ctypes.c_int, ctypes.c_int, _dp, vp]
    lib.gbsbin_moments.argtypes = [ctypes.POINTER(gbsbin_problem), vp, vp]
    lib.gbsbin_cumulants3.argtypes = [ctypes.POINTER(gbsbin_problem), vp]
    lib.gbsbin_cumulants3.restype = ctypes.c_int
    lib.gbsbin_cumulants4.argtypes = [ctypes.POINTER(gbsbin_problem), vp]
    lib.gbsbin_cumulants4.restype = ctypes.c_int
    lib.gbsbin_total_photon_series.argtypes = [ctypes.POINTER(gbsbin_problem), ctypes.c_int, vp]
    lib.gbsbin_total_photon_series.restype = ctypes.c_int
    lib.gbsbin_cumulant_groups.argtypes = [ctypes.POINTER(gbsbin_problem), ctypes.c_uint, vp]
    lib.gbsbin_cumulant_groups.restype = ctypes.c_int
    lib.gbsbin_prob_distinguishable.argtypes = [ctypes.POINTER(gbsbin_problem), _ip, vp, vp]
    lib.gbsbin_prob_distinguishable.restype = ctypes.c_int
    lib.gbsbin_prob_distinguishable_device.argtypes = [ctypes.POINTER(gbsbin_problem), _ip, vp, vp, vp]
    lib.gbsbin_prob_distinguishable_device.restype = ctypes.c_int
    lib.gbsbin_cumulants_device.argtypes = [ctypes.POINTER(gbsbin_problem), ctypes.c_int, vp, vp, vp, vp, vp, vp]
    lib.gbsbin_cumulants_device.restype = ctypes.c_int
    lib.gbsbin_read_points.argtypes = [vp, vp, vp, vp]
    lib.gbsbin_table_from_logq_noalloc.argtypes = [ctypes.c_int, _ip, ctypes.c_int, vp, vp, vp]
    lib.gbsbin_backward.argtypes = [vp, vp, ctypes.POINTER(gbsbin_grads), vp]
    lib.gbsbin_backward_device.argtypes = [vp, vp, vp, vp, vp]
    lib.gbsbin_backward_device.restype = ctypes.c_int
    lib.gbsbin_autotune.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _ip, _dp]
    lib.gbsbin_batch_create.argtypes = [ctypes.POINTER(gbsbin_problem), ctypes.c_int, ctypes.POINTER(gbsbin_options),
                                        ctypes.c_int, ctypes.POINTER(vp)]
    lib.gbsbin_batch_execute.argtypes = [vp, ctypes.POINTER(vp), vp]
    lib.gbsbin_batch_capture_graph.argtypes = [vp, ctypes.POINTER(vp), vp]
    lib.gbsbin_batch_replay.argtypes = [vp, vp]
    lib.gbsbin_batch_table_size.argtypes = [vp, ctypes.c_int]
    lib.gbsbin_batch_table_size.restype = ctypes.c_longlong
    lib.gbsbin_batch_diagnostics.argtypes = [vp, ctypes.c_int, ctypes.POINTER(gbsbin_diag), vp]
    lib.gbsbin_batch_read_points.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.gbsbin_batch_destroy.argtypes = [vp]
    lib.gbsbin_fock_plan_create.argtypes = [ctypes.POINTER(gbsbin_fock_problem), ctypes.POINTER(gbsbin_options),
                                            ctypes.POINTER(vp)]
    lib.gbsbin_fock_plan_set_transfer.argtypes = [vp, _cp, vp]
    lib.gbsbin_fock_plan_table_size.argtypes = [vp]
    lib.gbsbin_fock_plan_table_size.restype = ctypes.c_longlong
    lib.gbsbin_fock_plan_nodes.argtypes = [vp]
    lib.gbsbin_fock_plan_nodes.restype = ctypes.c_longlong
    lib.gbsbin_fock_execute.argtypes = [vp, vp, vp]
    lib.gbsbin_fock_execute_host.argtypes = [vp, vp, vp]
    lib.gbsbin_fock_diagnostics.argtypes = [vp, ctypes.POINTER(gbsbin_diag), vp]
    lib.gbsbin_fock_plan_destroy.argtypes = [vp]
    hp = ctypes.POINTER(gbsbin_herald_problem)
    lib.gbsbin_herald_plan_create.argtypes = [hp, ctypes.POINTER(gbsbin_options), ctypes.POINTER(vp)]
    lib.gbsbin_herald_table_size.argtypes = [vp]
    lib.gbsbin_herald_table_size.restype = ctypes.c_longlong
    lib.gbsbin_herald_prob_size.argtypes = [vp]
    lib.gbsbin_herald_prob_size.restype = ctypes.c_longlong
    lib.gbsbin_herald_execute.argtypes = [vp, vp, vp, vp]
    lib.gbsbin_herald_execute_host.argtypes = [vp, vp, vp, vp]
    lib.gbsbin_herald_diagnostics.argtypes = [vp, ctypes.POINTER(gbsbin_diag), vp]
    lib.gbsbin_herald_plan_destroy.argtypes = [vp]
    for f in ("gbsbin_herald_plan_create", "gbsbin_herald_execute", "gbsbin_herald_execute_host",
              "gbsbin_herald_diagnostics", "gbsbin_herald_plan_destroy"):
        getattr(lib, f).restype = ctypes.c_int
    for f in ("gbsbin_plan_create", "gbsbin_plan_set_state", "gbsbin_plan_destroy", "gbsbin_execute",
              "gbsbin_execute_host", "gbsbin_execute_host_async", "gbsbin_diagnostics", "gbsbin_alu_peak",
              "gbsbin_read_points",
              "gbsbin_table_from_logq_noalloc", "gbsbin_backward", "gbsbin_autotune", "gbsbin_batch_create",
              "gbsbin_batch_execute", "gbsbin_batch_capture_graph", "gbsbin_batch_replay",
              "gbsbin_batch_diagnostics", "gbsbin_batch_read_points", "gbsbin_batch_destroy",
              "gbsbin_fock_plan_create", "gbsbin_fock_plan_set_transfer", "gbsbin_fock_execute",
              "gbsbin_fock_execute_host", "gbsbin_fock_diagnostics", "gbsbin_fock_plan_destroy"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status, where):
    if status != 0:
        raise GbsbinError(status, where)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(buf):
    if isinstance(buf, int):
        return ctypes.c_void_p(buf)
    if isinstance(buf, np.ndarray):
        return ctypes.c_void_p(buf.ctypes.data)
    return ctypes.c_void_p(buf.data_ptr())


class ProblemArgs:
    """Marshals a problem description (any object with M, K, r, T, bin_of_mode, cutoff and
    optional alpha, V, sigma1, zbar attributes) into a gbsbin_problem; keeps the arrays alive."""

    def __init__(self, prob):
        def carr(a):
            if a is None:
                return None, None
            arr = np.ascontiguousarray(np.asarray(a, dtype=np.complex128).reshape(-1))
            return arr, arr.ctypes.data_as(_cp)

        self.M, self.K = int(prob.M), int(prob.K)
        self._keep = []
        sig = getattr(prob, "sigma1", None)
        self.r = None if getattr(prob, "r", None) is None else \
            np.ascontiguousarray(np.asarray(prob.r, dtype=np.float64).reshape(-1))
        T, Tp = carr(getattr(prob, "T", None))
        al, alp = carr(getattr(prob, "alpha", None))
        V, Vp = carr(getattr(prob, "V", None))
        S, Sp = carr(sig)
        Z, Zp = carr(getattr(prob, "zbar", None))
        self.bins = np.ascontiguousarray(np.asarray(prob.bin_of_mode, dtype=np.int32))
        self.cut = np.ascontiguousarray(np.asarray(prob.cutoff, dtype=np.int32))
        self._keep += [T, al, V, S, Z]
        self.c = gbsbin_problem(
            self.M, self.K, None if self.r is None else self.r.ctypes.data_as(_dp), Tp, alp, Vp, Sp, Zp,
            self.bins.ctypes.data_as(_ip), int(len(self.cut)), self.cut.ctypes.data_as(_ip))


def gbsbin_default_options():
    o = gbsbin_options()
    load().gbsbin_default_options(ctypes.byref(o))
    return o


def make_options(precision=GBSBIN_FP64, oversample=1, want_diagnostics=True, tile_override=0,
                 want_timing=False, want_backward=False, shard=None):
    o = gbsbin_default_options()
    o.precision, o.oversample = int(precision), int(oversample)
    o.want_diagnostics, o.tile_override = int(bool(want_diagnostics)), int(tile_override)
    o.want_timing = int(bool(want_timing))
    o.want_backward = int(bool(want_backward))
    if shard is not None:
        o.shard_begin, o.shard_end = int(shard[0]), int(shard[1])
    return o


def gbsbin_plan_create(prob, options=None):
    """Returns an opaque plan handle (ctypes.c_void_p)."""
    lib = load()
    args = prob if isinstance(prob, ProblemArgs) else ProblemArgs(prob)
    opt = options if options is not None else gbsbin_default_options()
    h = ctypes.c_void_p()
    _check(lib.gbsbin_plan_create(ctypes.byref(args.c), ctypes.byref(opt), ctypes.byref(h)), "gbsbin_plan_create")
    return h


def gbsbin_plan_set_state(plan, prob, stream=None):
    args = prob if isinstance(prob, ProblemArgs) else ProblemArgs(prob)
    _check(load().gbsbin_plan_set_state(plan, ctypes.byref(args.c), _stream_handle(stream)),
           "gbsbin_plan_set_state")


def gbsbin_plan_destroy(plan):
    _check(load().gbsbin_plan_destroy(plan), "gbsbin_plan_destroy")


def gbsbin_plan_table_size(plan):
    return int(load().gbsbin_plan_table_size(plan))


def gbsbin_execute(plan, P_out, stream=None):
    """P_out: device buffer (torch CUDA float64 tensor or raw pointer) of table_size doubles."""
    _check(load().gbsbin_execute(plan, _ptr(P_out), _stream_handle(stream)), "gbsbin_execute")


def gbsbin_execute_host(plan, P_out_host, stream=None):
    """P_out_host: host float64 buffer (numpy array, pinned torch tensor or pointer)."""
    _check(load().gbsbin_execute_host(plan, _ptr(P_out_host), _stream_handle(stream)), "gbsbin_execute_host")


def gbsbin_execute_host_async(plan, P_out_host, stream=None):
    """Enqueue the execute and the copy into P_out_host (pinned host buffer) and return;
    synchronise the stream before reading P_out_host."""
    _check(load().gbsbin_execute_host_async(plan, _ptr(P_out_host), _stream_handle(stream)),
           "gbsbin_execute_host_async")


def gbsbin_diagnostics(plan, stream=None):
    """Returns (status, dict); status is GBSBIN_ERR_NUMERIC (7) if any point had a bad pivot."""
    d = gbsbin_diag()
    st = load().gbsbin_diagnostics(plan, ctypes.byref(d), _stream_handle(stream))
    out = {f: getattr(d, f) for f, _ in gbsbin_diag._fields_}
    out["kernel_name"] = KERNELS.get(out["kernel"], "?")
    if st not in (0, 7):
        raise GbsbinError(st, "gbsbin_diagnostics")
    return st, out


def gbsbin_read_points(plan, n_evaluated, stream=None):
    """Returns (logq complex128 (n_evaluated,), min pivot float64 (n_evaluated,))."""
    lq = np.zeros(int(n_evaluated), dtype=np.complex128)
    mp = np.zeros(int(n_evaluated), dtype=np.float64)
    _check(load().gbsbin_read_points(plan, _ptr(lq), _ptr(mp), _stream_handle(stream)), "gbsbin_read_points")
    return lq, mp


def evaluated_point_digits(cutoff, oversample=1):
    """Digits k (n_evaluated, L) of the evaluated half grid, in the library's order."""
    radix = [oversample * (int(c) + 1) for c in cutoff]
    half = radix[-1] // 2 + 1
    axes = [np.arange(r) for r in radix[:-1]] + [np.arange(half)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], axis=1)


def gbsbin_table_from_logq_noalloc(cutoff, oversample, logq_dev, P_out, stream=None):
    """Table from per-point log q (device buffer of n_evaluated complex values) into P_out
    (device), using the library's fixed scratch instead of allocating."""
    cut = np.ascontiguousarray(np.asarray(cutoff, dtype=np.int32))
    _check(load().gbsbin_table_from_logq_noalloc(int(len(cut)), cut.ctypes.data_as(_ip), int(oversample),
                                                 _ptr(logq_dev), _ptr(P_out), _stream_handle(stream)),
           "gbsbin_table_from_logq_noalloc")


def gbsbin_backward(plan, dL_dP, M, K, n, stream=None, want=("r", "T", "alpha", "V", "sigma1", "zbar")):
    """Reverse pass: dL_dP is a device buffer of table_size doubles.  Returns a dict of
    numpy arrays (complex gradients as dL/dRe + i dL/dIm) for the names in ``want``."""
    shapes = {"r": (M * K,), "T": (M * M,), "alpha": (M * K,), "V": (M * K * K,), "sigma1": (n * n,),
              "zbar": (n,)}
    out = {k: np.zeros(shapes[k], dtype=np.float64 if k == "r" else np.complex128) for k in want}
    g = gbsbin_grads()
    for k, arr in out.items():
        ptr = arr.ctypes.data_as(_dp if k == "r" else _cp)
        setattr(g, "d_" + k, ptr)
    _check(load().gbsbin_backward(plan, _ptr(dL_dP), ctypes.byref(g), _stream_handle(stream)), "gbsbin_backward")
    res = {k: v for k, v in out.items()}
    if "T" in res:
        res["T"] = res["T"].reshape(M, M)
    if "r" in res:
        res["r"] = res["r"].reshape(M, K)
    if "alpha" in res:
        res["alpha"] = res["alpha"].reshape(M, K)
    if "V" in res:
        res["V"] = res["V"].reshape(M, K, K)
    if "sigma1" in res:
        res["sigma1"] = res["sigma1"].reshape(n, n)
    return res


def gbsbin_backward_device(plan, dL_dP, dL_dXA, dL_dgamma, stream=None):
    """Asynchronous reverse pass to the adjacency adjoints S (n x n) and s (n), device buffers
    of complex128: dL = Re(sum S_ij dXA_ij + sum s_i dgamma_i)."""
    _check(load().gbsbin_backward_device(plan, _ptr(dL_dP), _ptr(dL_dXA), _ptr(dL_dgamma), _stream_handle(stream)),
           "gbsbin_backward_device")


def gbsbin_autotune(n, precision):
    """Returns (kernel id, points per CTA, microseconds per evaluated point)."""
    k, p, us = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(load().gbsbin_autotune(int(n), int(precision), ctypes.byref(k), ctypes.byref(p), ctypes.byref(us)),
           "gbsbin_autotune")
    return k.value, p.value, us.value


def gbsbin_strerror(status):
    return load().gbsbin_strerror(int(status)).decode()


def gbsbin_moments(prob):
    """Exact mean (L,) and covariance (L, L) of the binned counts (host, FP64, no device)."""
    args = prob if isinstance(prob, ProblemArgs) else ProblemArgs(prob)
    L = len(np.asarray(prob.cutoff))
    mean = np.zeros(L)
    cov = np.zeros((L, L))
    _check(load().gbsbin_moments(ctypes.byref(args.c), mean.ctypes.data_as(ctypes.c_void_p),
                                 cov.ctypes.data_as(ctypes.c_void_p)), "gbsbin_moments")
    return mean, cov


def gbsbin_cumulants3(prob):
    """Exact third cumulants kappa_lmn of the binned counts (host FP64), an (L, L, L) array."""
    args = ProblemArgs(prob)
    L = int(len(args.cut))
    k3 = np.zeros((L, L, L), dtype=np.float64)
    _check(load().gbsbin_cumulants3(ctypes.byref(args.c), k3.ctypes.data_as(ctypes.c_void_p)), "gbsbin_cumulants3")
    return k3


def gbsbin_cumulants4(prob):
    """Exact fourth cumulants kappa_{l1 l2 l3 l4} of the binned counts (host FP64), an
    (L, L, L, L) array."""
    args = ProblemArgs(prob)
    L = int(len(args.cut))
    k4 = np.zeros((L, L, L, L), dtype=np.float64)
    _check(load().gbsbin_cumulants4(ctypes.byref(args.c), k4.ctypes.data_as(ctypes.c_void_p)), "gbsbin_cumulants4")
    return k4


def gbsbin_cumulants_device(prob, order=4, precision=GBSBIN_FP64, stream=None, with_time=False):
    """Cumulant tensors of orders 1..order of the binned counts on the GPU (FP64, or the
    products in pairs of FP32 with GBSBIN_FP32_REFINE): the list [mean (L,), cov (L, L),
    k3 (L, L, L), k4 (L, L, L, L)][:order]; with_time also returns the device time of the
    launches in ms."""
    if not 1 <= int(order) <= 4:
        raise ValueError("order must be 1..4")
    args = ProblemArgs(prob)
    L = int(len(args.cut))
    outs = [np.zeros((L,) * r, dtype=np.float64) for r in range(1, int(order) + 1)]
    ptrs = [o.ctypes.data_as(ctypes.c_void_p) for o in outs] + [None] * (4 - len(outs))
    ms = ctypes.c_double()
    _check(load().gbsbin_cumulants_device(ctypes.byref(args.c), int(precision), *ptrs, ctypes.byref(ms),
                                          _stream_handle(stream)),
           "gbsbin_cumulants_device")
    return (outs, ms.value) if with_time else outs


def gbsbin_total_photon_series(prob, Nmax):
    """Total photon-number distribution Pr(N), N = 0..Nmax, by the power series (host FP64)."""
    args = ProblemArgs(prob)
    out = np.zeros(int(Nmax) + 1, dtype=np.float64)
    _check(load().gbsbin_total_photon_series(ctypes.byref(args.c), int(Nmax), out.ctypes.data_as(ctypes.c_void_p)),
           "gbsbin_total_photon_series")
    return out


def gbsbin_cumulant_groups(prob, groups):
    """Joint cumulant of the counts of the distinct groups in `groups` (the coarse-grained loop
    Montrealer; host FP64)."""
    mask = 0
    for g in groups:
        if mask >> int(g) & 1:
            raise ValueError("groups must be distinct")
        mask |= 1 << int(g)
    args = ProblemArgs(prob)
    out = ctypes.c_double()
    _check(load().gbsbin_cumulant_groups(ctypes.byref(args.c), ctypes.c_uint(mask), ctypes.byref(out)),
           "gbsbin_cumulant_groups")
    return out.value


GBSBIN_ERR_PRECISION = 10


def _dist_result(status, where, out, err, with_error):
    """Value (and error estimate) of an App. D call; a result that lost its digits to
    cancellation raises GbsbinError(GBSBIN_ERR_PRECISION) carrying ``value`` and ``abs_err``."""
    if status == GBSBIN_ERR_PRECISION:
        e = GbsbinError(status, where)
        e.value, e.abs_err = out.value, err.value
        raise e
    _check(status, where)
    return (out.value, err.value) if with_error else out.value


def gbsbin_prob_distinguishable(prob, pattern, with_error=False):
    """Fine-grained Pr(n) of an undisplaced state with fully distinguishable internal modes
    (App. D; host FP64).  with_error: also return the estimate of its absolute rounding error."""
    pat = np.ascontiguousarray(np.asarray(pattern, dtype=np.int32))
    args = ProblemArgs(prob)
    out, err = ctypes.c_double(), ctypes.c_double()
    st = load().gbsbin_prob_distinguishable(ctypes.byref(args.c), pat.ctypes.data_as(_ip), ctypes.byref(out),
                                            ctypes.byref(err))
    return _dist_result(st, "gbsbin_prob_distinguishable", out, err, with_error)


def gbsbin_prob_distinguishable_device(prob, pattern, stream=None, with_error=False):
    """gbsbin_prob_distinguishable with the sum over the evaluation points on the GPU."""
    pat = np.ascontiguousarray(np.asarray(pattern, dtype=np.int32))
    args = ProblemArgs(prob)
    out, err = ctypes.c_double(), ctypes.c_double()
    st = load().gbsbin_prob_distinguishable_device(ctypes.byref(args.c), pat.ctypes.data_as(_ip), ctypes.byref(out),
                                                   ctypes.byref(err), _stream_handle(stream))
    return _dist_result(st, "gbsbin_prob_distinguishable_device", out, err, with_error)


def gbsbin_alu_peak(precision, blocks, stream=None):
    v = ctypes.c_double()
    _check(load().gbsbin_alu_peak(int(precision), int(blocks), ctypes.byref(v), _stream_handle(stream)),
           "gbsbin_alu_peak")
    return v.value


class Plan:
    """Owning wrapper: ``with Plan(prob, precision=...) as p: P = p.table()``."""

    def __init__(self, prob, precision=GBSBIN_FP64, oversample=1, want_diagnostics=True, tile_override=0,
                 want_timing=False, want_backward=False, shard=None):
        """shard = (begin, end): evaluate only points [begin, end) of the evaluated half grid
        (plus point 0 for the normalisation); table() then returns their partial table."""
        self.options = make_options(precision, oversample, want_diagnostics, tile_override, want_timing,
                                    want_backward, shard)
        self.handle = gbsbin_plan_create(prob, self.options)
        self.shape = tuple(int(c) + 1 for c in prob.cutoff)
        self.M, self.K = int(prob.M), int(prob.K)
        self.n = 2 * self.M * self.K

    def backward(self, dL_dP, stream=None, want=("r", "T", "alpha", "V", "sigma1", "zbar")):
        """Gradients of L for the plan's current state given dL/dP (CUDA float64 tensor)."""
        return gbsbin_backward(self.handle, dL_dP, self.M, self.K, self.n, stream, want)

    def backward_device(self, dL_dP, stream=None):
        """Adjacency adjoints (S, s) as new CUDA complex128 tensors, asynchronously."""
        import torch
        S = torch.empty((self.n, self.n), dtype=torch.complex128, device="cuda")
        g = torch.empty((self.n,), dtype=torch.complex128, device="cuda")
        gbsbin_backward_device(self.handle, dL_dP, S, g, stream)
        return S, g

    def table(self, stream=None):
        """Execute into a new CUDA float64 tensor shaped (N_1+1, ..., N_L+1)."""
        import torch
        out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        gbsbin_execute(self.handle, out, stream)
        return out

    def diagnostics(self, stream=None):
        return gbsbin_diagnostics(self.handle, stream)

    def close(self):
        if self.handle is not None:
            gbsbin_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _State:
    """Physical description assembled from tensors for one evaluation."""

    def __init__(self, template, r, T, alpha, V):
        self.M, self.K = template.M, template.K
        self.bin_of_mode, self.cutoff = template.bin_of_mode, template.cutoff
        self.r = r.detach().cpu().numpy()
        self.T = T.detach().cpu().numpy()
        self.alpha = None if alpha is None else alpha.detach().cpu().numpy()
        self.V = None if V is None else V.detach().cpu().numpy()


def _autograd_function():
    import torch

    class BinnedDistribution(torch.autograd.Function):
        """P(b) as a differentiable function of (r, T, alpha, V) through a plan created with
        want_backward; the reverse pass is gbsbin_backward."""

        @staticmethod
        def forward(ctx, plan, template, r, T, alpha, V):
            gbsbin_plan_set_state(plan.handle, _State(template, r, T, alpha, V))
            P = plan.table()
            ctx.plan = plan
            ctx.has = (alpha is not None, V is not None)
            ctx.dev = (r.device, T.device)
            return P

        @staticmethod
        def backward(ctx, grad_P):
            g = ctx.plan.backward(grad_P.detach().contiguous().to(torch.float64),
                                  want=("r", "T", "alpha", "V"))
            d_r = torch.from_numpy(g["r"]).to(ctx.dev[0])
            d_T = torch.from_numpy(g["T"]).to(ctx.dev[1])
            d_a = torch.from_numpy(g["alpha"]).to(ctx.dev[0]) if ctx.has[0] else None
            d_V = torch.from_numpy(g["V"]).to(ctx.dev[0]) if ctx.has[1] else None
            return None, None, d_r, d_T, d_a, d_V

    return BinnedDistribution


_BD = None


def binned_distribution(plan, template, r, T, alpha=None, V=None):
    """Differentiable binned table: ``plan`` is a :class:`Plan` made with want_backward for a
    problem with the same M, K, grouping and cutoffs as ``template``; r (float64, (M, K)),
    T (complex128, (M, M)), alpha (complex128, (M, K)) and V (complex128, (M, K, K)) are
    torch tensors.  Returns a CUDA float64 tensor shaped (N_1+1, ..., N_L+1)."""
    global _BD
    if _BD is None:
        _BD = _autograd_function()
    return _BD.apply(plan, template, r, T, alpha, V)


class Batch:
    """Owning wrapper of a gbsbin batch: ``Batch(problems, precision=..., autotune=True)``."""

    def __init__(self, problems, precision=GBSBIN_FP64, oversample=1, want_diagnostics=True, tile_override=0,
                 autotune=False):
        self._args = [ProblemArgs(p) for p in problems]
        arr = (gbsbin_problem * len(self._args))(*[a.c for a in self._args])
        self.options = make_options(precision, oversample, want_diagnostics, tile_override)
        h = ctypes.c_void_p()
        _check(load().gbsbin_batch_create(arr, len(self._args), ctypes.byref(self.options), int(bool(autotune)),
                                          ctypes.byref(h)), "gbsbin_batch_create")
        self.handle = h
        self.shapes = [tuple(int(c) + 1 for c in p.cutoff) for p in problems]
        self.outputs = None

    def _out_array(self, outs):
        return (ctypes.c_void_p * len(outs))(*[o.data_ptr() for o in outs])

    def allocate(self):
        import torch
        self.outputs = [torch.empty(s, dtype=torch.float64, device="cuda") for s in self.shapes]
        return self.outputs

    def execute(self, stream=None):
        """Evaluate every table into self.outputs (allocated on first use)."""
        if self.outputs is None:
            self.allocate()
        _check(load().gbsbin_batch_execute(self.handle, self._out_array(self.outputs), _stream_handle(stream)),
               "gbsbin_batch_execute")
        return self.outputs

    def capture(self, stream):
        if self.outputs is None:
            self.allocate()
        _check(load().gbsbin_batch_capture_graph(self.handle, self._out_array(self.outputs), _stream_handle(stream)),
               "gbsbin_batch_capture_graph")

    def replay(self, stream):
        _check(load().gbsbin_batch_replay(self.handle, _stream_handle(stream)), "gbsbin_batch_replay")
        return self.outputs

    def diagnostics(self, i, stream=None):
        d = gbsbin_diag()
        st = load().gbsbin_batch_diagnostics(self.handle, int(i), ctypes.byref(d), _stream_handle(stream))
        if st not in (0, 7):
            raise GbsbinError(st, "gbsbin_batch_diagnostics")
        out = {f: getattr(d, f) for f, _ in gbsbin_diag._fields_}
        out["kernel_name"] = KERNELS.get(out["kernel"], "?")
        return st, out

    def read_points(self, i, n_evaluated, stream=None):
        lq = np.zeros(int(n_evaluated), dtype=np.complex128)
        mp = np.zeros(int(n_evaluated), dtype=np.float64)
        _check(load().gbsbin_batch_read_points(self.handle, int(i), _ptr(lq), _ptr(mp), _stream_handle(stream)),
               "gbsbin_batch_read_points")
        return lq, mp

    def close(self):
        if getattr(self, "handle", None) is not None:
            _check(load().gbsbin_batch_destroy(self.handle), "gbsbin_batch_destroy")
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ Fock inputs (App. C)
class FockProblemArgs:
    """Marshals a Fock-input problem (M, T, photons, bin_of_mode, cutoff) into a
    gbsbin_fock_problem; keeps the arrays alive."""

    def __init__(self, prob):
        self.M = int(prob.M)
        self.T = np.ascontiguousarray(np.asarray(prob.T, dtype=np.complex128).reshape(-1))
        self.photons = np.ascontiguousarray(np.asarray(prob.photons, dtype=np.int32))
        self.bins = np.ascontiguousarray(np.asarray(prob.bin_of_mode, dtype=np.int32))
        self.cut = np.ascontiguousarray(np.asarray(prob.cutoff, dtype=np.int32))
        self.c = gbsbin_fock_problem(self.M, self.T.ctypes.data_as(_cp), self.photons.ctypes.data_as(_ip),
                                     self.bins.ctypes.data_as(_ip), int(len(self.cut)), self.cut.ctypes.data_as(_ip))


def gbsbin_fock_plan_create(prob, options=None):
    lib = load()
    args = FockProblemArgs(prob)
    opts = options if options is not None else gbsbin_default_options()
    h = ctypes.c_void_p()
    _check(lib.gbsbin_fock_plan_create(ctypes.byref(args.c), ctypes.byref(opts), ctypes.byref(h)),
           "gbsbin_fock_plan_create")
    return h


def gbsbin_fock_plan_set_transfer(plan, T, stream=None):
    arr = np.ascontiguousarray(np.asarray(T, dtype=np.complex128).reshape(-1))
    _check(load().gbsbin_fock_plan_set_transfer(plan, arr.ctypes.data_as(_cp), _stream_handle(stream)),
           "gbsbin_fock_plan_set_transfer")


def gbsbin_fock_plan_table_size(plan):
    return int(load().gbsbin_fock_plan_table_size(plan))


def gbsbin_fock_execute(plan, P_out, stream=None):
    _check(load().gbsbin_fock_execute(plan, _ptr(P_out), _stream_handle(stream)), "gbsbin_fock_execute")


def gbsbin_fock_execute_host(plan, P_out_host, stream=None):
    _check(load().gbsbin_fock_execute_host(plan, _ptr(P_out_host), _stream_handle(stream)),
           "gbsbin_fock_execute_host")


def gbsbin_fock_diagnostics(plan, stream=None):
    d = gbsbin_diag()
    st = load().gbsbin_fock_diagnostics(plan, ctypes.byref(d), _stream_handle(stream))
    out = {f: getattr(d, f) for f, _ in gbsbin_diag._fields_}
    out["kernel_name"] = KERNELS.get(out["kernel"], "?")
    out["status"] = st
    return out


def gbsbin_fock_plan_destroy(plan):
    _check(load().gbsbin_fock_plan_destroy(plan), "gbsbin_fock_plan_destroy")


class FockPlan:
    """Owning wrapper for Fock inputs: ``with FockPlan(prob) as p: P = p.table()``.

    precision GBSBIN_FP64 runs the FP64 kernel, GBSBIN_FP32_REFINE the FP32-pair kernel."""

    def __init__(self, prob, precision=GBSBIN_FP64, oversample=1, want_diagnostics=True, tile_override=0,
                 want_timing=False, shard=None):
        """shard = (begin, end): walk only the input nodes [begin, end) (Gray-code order);
        table() then returns their partial table."""
        self.options = make_options(precision, oversample, want_diagnostics, tile_override, want_timing,
                                    shard=shard)
        self.handle = gbsbin_fock_plan_create(prob, self.options)
        self.shape = tuple(int(c) + 1 for c in prob.cutoff)

    def nodes(self):
        """Input nodes of the whole problem."""
        return int(load().gbsbin_fock_plan_nodes(self.handle))

    def set_transfer(self, T, stream=None):
        gbsbin_fock_plan_set_transfer(self.handle, T, stream)

    def table(self, stream=None):
        """Execute into a new CUDA float64 tensor shaped (N_1+1, ..., N_L+1)."""
        import torch
        out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        gbsbin_fock_execute(self.handle, out, stream)
        return out

    def table_host(self, stream=None):
        out = np.empty(self.shape, dtype=np.float64)
        gbsbin_fock_execute_host(self.handle, out, stream)
        return out

    def diagnostics(self, stream=None):
        return gbsbin_fock_diagnostics(self.handle, stream)

    def close(self):
        if self.handle is not None:
            gbsbin_fock_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ heralded states (Sec. VII)
class HeraldProblemArgs:
    """Marshals a state (M, K and r, T, optional alpha, V - or sigma1, optional zbar), the
    per-mode roles (heralding group >= 0, GBSBIN_HERALD_TRACED, GBSBIN_HERALD_KEPT), the
    heralding cutoffs and the kept modes' Fock cutoff into a gbsbin_herald_problem."""

    class _State:
        def __init__(self, st):
            self.__dict__.update({k: getattr(st, k, None) for k in ("M", "K", "r", "T", "alpha", "V", "sigma1",
                                                                     "zbar")})
            self.bin_of_mode = [0] * int(st.M)     # ignored by the library
            self.cutoff = [0]

    def __init__(self, state, roles, cutoff, fock_cutoff):
        self.state = ProblemArgs(self._State(state))
        self.roles = np.ascontiguousarray(np.asarray(roles, dtype=np.int32))
        self.cut = np.ascontiguousarray(np.asarray(cutoff, dtype=np.int32))
        self.c = gbsbin_herald_problem(self.state.c, self.roles.ctypes.data_as(_ip), int(len(self.cut)),
                                       self.cut.ctypes.data_as(_ip), int(fock_cutoff))


def gbsbin_herald_plan_create(state, roles, cutoff, fock_cutoff, options=None):
    args = HeraldProblemArgs(state, roles, cutoff, fock_cutoff)
    opts = options if options is not None else gbsbin_default_options()
    h = ctypes.c_void_p()
    _check(load().gbsbin_herald_plan_create(ctypes.byref(args.c), ctypes.byref(opts), ctypes.byref(h)),
           "gbsbin_herald_plan_create")
    return h


def gbsbin_herald_table_size(plan):
    return int(load().gbsbin_herald_table_size(plan))


def gbsbin_herald_prob_size(plan):
    return int(load().gbsbin_herald_prob_size(plan))


def gbsbin_herald_execute(plan, rho_out, prob_out, stream=None):
    _check(load().gbsbin_herald_execute(plan, _ptr(rho_out), _ptr(prob_out), _stream_handle(stream)),
           "gbsbin_herald_execute")


def gbsbin_herald_execute_host(plan, rho_host, prob_host, stream=None):
    _check(load().gbsbin_herald_execute_host(plan, _ptr(rho_host), _ptr(prob_host), _stream_handle(stream)),
           "gbsbin_herald_execute_host")


def gbsbin_herald_diagnostics(plan, stream=None):
    d = gbsbin_diag()
    st = load().gbsbin_herald_diagnostics(plan, ctypes.byref(d), _stream_handle(stream))
    out = {f: getattr(d, f) for f, _ in gbsbin_diag._fields_}
    out["kernel_name"] = KERNELS.get(out["kernel"], "?")
    out["status"] = st
    return out


def gbsbin_herald_plan_destroy(plan):
    _check(load().gbsbin_herald_plan_destroy(plan), "gbsbin_herald_plan_destroy")


class HeraldPlan:
    """Owning wrapper: ``with HeraldPlan(state, roles, cutoff, fock_cutoff) as h: rho, pr = h.states()``.

    ``rho[b..., u..., v...] = <v| rho(b) |u>`` (unnormalised; ``pr[b]`` = Pr(b) its trace over all
    kept photon numbers)."""

    def __init__(self, state, roles, cutoff, fock_cutoff, oversample=1, want_timing=False):
        self.options = make_options(GBSBIN_FP64, oversample, True, 0, want_timing)
        self.handle = gbsbin_herald_plan_create(state, roles, cutoff, fock_cutoff, self.options)
        nk = int(sum(1 for r in roles if int(r) == GBSBIN_HERALD_KEPT))
        self.prob_shape = tuple(int(c) + 1 for c in cutoff)
        self.shape = self.prob_shape + (int(fock_cutoff) + 1,) * (2 * nk)

    def states(self, stream=None):
        """Execute into new CUDA tensors: rho (complex128, ``shape``) and Pr(b) (float64)."""
        import torch
        rho = torch.empty(self.shape, dtype=torch.complex128, device="cuda")
        pr = torch.empty(self.prob_shape, dtype=torch.float64, device="cuda")
        gbsbin_herald_execute(self.handle, rho, pr, stream)
        return rho, pr

    def states_host(self, stream=None):
        rho = np.empty(self.shape, dtype=np.complex128)
        pr = np.empty(self.prob_shape, dtype=np.float64)
        gbsbin_herald_execute_host(self.handle, rho, pr, stream)
        return rho, pr

    def diagnostics(self, stream=None):
        return gbsbin_herald_diagnostics(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None) is not None:
            gbsbin_herald_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
