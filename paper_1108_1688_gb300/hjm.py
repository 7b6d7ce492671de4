"""Thin ctypes binding of libhjm (include/hjm.h): same names, argument
marshalling only. Every step of the pricing path runs in the library's CUDA
kernels; there is no Python or CPU fallback, and importing this module fails
loudly when the compiled library is missing.

Structs mirror the C header field by field. Item dicts (curve, model, grid,
inst), as produced by paper_1108_1688_gb300.workloads, convert with
`batch_item(d)`; the field `lambda` of the model struct is spelled `lambda_`
here because `lambda` is a Python keyword.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhjm.so")

HJM_OK, HJM_EINVAL, HJM_ENOMEM, HJM_ECUDA, HJM_ETOL, HJM_ETIMEOUT, HJM_ENUMERIC, HJM_ERANGE = range(8)
HJM_FP64, HJM_FP32, HJM_MIXED = 0, 1, 2
HJM_CURVE_FLAT, HJM_CURVE_NELSON_SIEGEL, HJM_CURVE_KNOTS = 0, 1, 2
HJM_SCHEME_DOUGLAS, HJM_SCHEME_CS, HJM_SCHEME_MCS, HJM_SCHEME_HV = 0, 1, 2, 3
HJM_ZCB, HJM_CAPLET, HJM_FLOORLET = 0, 1, 2

PRECISIONS = {"fp64": HJM_FP64, "fp32": HJM_FP32, "mixed": HJM_MIXED,
              HJM_FP64: HJM_FP64, HJM_FP32: HJM_FP32, HJM_MIXED: HJM_MIXED}


HJM_MAX_KNOTS = 32
HJM_LINES_TMA = 15  # p2_warps / p3_warps: strided lines moved by the Tensor Memory Accelerator


class hjm_curve(C.Structure):
    _fields_ = [("kind", C.c_int), ("flat_rate", C.c_double), ("beta0", C.c_double),
                ("beta1", C.c_double), ("beta2", C.c_double), ("tau", C.c_double),
                ("n_knots", C.c_int), ("knot_t", C.c_double * HJM_MAX_KNOTS),
                ("knot_P", C.c_double * HJM_MAX_KNOTS)]


class hjm_model_params(C.Structure):
    _fields_ = [("kappa", C.c_double), ("lambda_", C.c_double), ("gamma", C.c_double),
                ("theta", C.c_double), ("epsilon", C.c_double), ("rho", C.c_double),
                ("v0", C.c_double)]


class hjm_grid_spec(C.Structure):
    _fields_ = [("n_r", C.c_int), ("n_y", C.c_int), ("n_v", C.c_int), ("n_steps", C.c_int),
                ("r_min", C.c_double), ("r_max", C.c_double), ("y_max", C.c_double),
                ("v_max", C.c_double), ("alpha_r", C.c_double), ("alpha_y", C.c_double),
                ("alpha_v", C.c_double), ("k_r", C.c_double), ("k_v", C.c_double),
                ("center_r_on_strike", C.c_int), ("theta_adi", C.c_double),
                ("y_boundary_order", C.c_int), ("explicit_midpoint", C.c_int), ("scheme", C.c_int)]


class hjm_instrument(C.Structure):
    _fields_ = [("kind", C.c_int), ("expiry_T", C.c_double), ("pay_TM", C.c_double),
                ("strike_K", C.c_double), ("strike_atm_relative", C.c_int)]


class hjm_price_info(C.Structure):
    _fields_ = [("precision_used", C.c_int), ("escalated", C.c_int), ("err_estimate", C.c_double),
                ("n_steps", C.c_int), ("time_us", C.c_float), ("tile_cfg", C.c_int), ("d_dr", C.c_double),
                ("d_dv", C.c_double)]


HJM_TRACE_KINDS = 6
TRACE_KIND_NAMES = ("setup", "terminal", "pass1", "pass2", "pass3", "readout")


class hjm_trace(C.Structure):
    _fields_ = [("launches", C.c_longlong * HJM_TRACE_KINDS), ("total_ms", C.c_double * HJM_TRACE_KINDS)]


class hjm_tile(C.Structure):
    _fields_ = [("p1_lanes", C.c_int), ("p1_nodes", C.c_int), ("p1_lines", C.c_int), ("p2_warps", C.c_int),
                ("p3_warps", C.c_int), ("p1_staged", C.c_int), ("p1_planes", C.c_int)]


class hjm_surrogate_cfg(C.Structure):
    _fields_ = [("n_train", C.c_size_t), ("hidden", C.c_int), ("depth", C.c_int), ("epochs", C.c_int),
                ("batch", C.c_int), ("lr", C.c_float), ("seed", C.c_uint64), ("box_lo", C.c_double * 9),
                ("box_hi", C.c_double * 9), ("label_grid", hjm_grid_spec), ("checkpoint_path", C.c_char_p)]


HJM_SURROGATE_PARAMS = 200193
HJM_SURROGATE_BINS = 72


class hjm_batch_item(C.Structure):
    _fields_ = [("curve", hjm_curve), ("model", hjm_model_params), ("grid", hjm_grid_spec),
                ("inst", hjm_instrument)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libhjm.so is not built (expected at %s); run "
                          "paper_1108_1688_gb300._build.build() first" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    P, vp, st = C.POINTER, C.c_void_p, C.c_int
    sig = {
        "hjm_grid_create": ([P(hjm_curve), P(hjm_model_params), P(hjm_grid_spec), vp, P(vp)], st),
        "hjm_grid_destroy": ([vp], st),
        "hjm_price": ([vp, P(hjm_instrument), st, C.c_double, P(C.c_double), P(hjm_price_info)], st),
        "hjm_price_batch": ([P(hjm_batch_item), C.c_size_t, st, C.c_double, vp, P(hjm_price_info), vp], st),
        "hjm_field": ([vp, P(hjm_instrument), st, C.c_int, vp], st),
        "hjm_axis": ([vp, P(hjm_instrument), C.c_int, vp, vp, vp], st),
        "hjm_douglas_pass": ([vp, P(hjm_instrument), st, C.c_int, C.c_int, vp, vp, vp], st),
        "hjm_price_static": ([P(hjm_batch_item), st, vp, vp], st),
        "hjm_surrogate_create": ([P(hjm_surrogate_cfg), vp, P(vp)], st),
        "hjm_surrogate_train": ([P(hjm_surrogate_cfg), vp, P(vp)], st),
        "hjm_surrogate_fit": ([vp, vp, vp, C.c_size_t, C.c_int, vp, P(C.c_float)], st),
        "hjm_surrogate_infer": ([vp, vp, C.c_size_t, vp, vp, vp], st),
        "hjm_surrogate_forward": ([vp, vp, C.c_size_t, vp, vp], st),
        "hjm_surrogate_loss_grad": ([vp, vp, vp, C.c_size_t, P(C.c_float), vp, vp], st),
        "hjm_surrogate_get_params": ([vp, vp], st),
        "hjm_surrogate_set_params": ([vp, vp], st),
        "hjm_surrogate_error_table": ([vp, vp], st),
        "hjm_surrogate_save": ([vp, C.c_char_p], st),
        "hjm_surrogate_load": ([C.c_char_p, P(vp)], st),
        "hjm_surrogate_destroy": ([vp], st),
        "hjm_mlp_gemm": ([C.c_int, C.c_int, C.c_int, vp, C.c_int, C.c_int, vp, C.c_int, C.c_int, vp, C.c_int, vp], st),
        "hjm_trace_enable": ([st], st),
        "hjm_trace_read": ([P(hjm_trace), st], st),
        "hjm_tile_get": ([C.c_int, C.c_int, C.c_int, st, P(hjm_tile)], st),
        "hjm_tile_set": ([C.c_int, C.c_int, C.c_int, st, P(hjm_tile)], st),
        "hjm_autotune": ([P(hjm_batch_item), C.c_size_t, st, C.c_int, vp], st),
        "hjm_wait_status": ([st], st),
        "hjm_surrogate_premium": ([vp, vp, C.c_size_t, vp, vp], st),
        "hjm_surrogate_gauss_premium": ([vp, C.c_size_t, vp, vp], st),
        "hjm_price_strip": ([P(hjm_batch_item), C.c_size_t, st, C.c_double, P(C.c_double), P(C.c_double), vp], st),
        "hjm_test_drop_plane": ([C.c_int, C.c_uint], st),
        "hjm_status_string": ([st], C.c_char_p),
        "hjm_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()
EXPORTED = ("hjm_grid_create", "hjm_grid_destroy", "hjm_price", "hjm_price_batch", "hjm_field",
            "hjm_axis", "hjm_douglas_pass", "hjm_price_static", "hjm_surrogate_create", "hjm_surrogate_train",
            "hjm_surrogate_fit", "hjm_surrogate_infer", "hjm_surrogate_forward", "hjm_surrogate_loss_grad",
            "hjm_surrogate_get_params", "hjm_surrogate_set_params", "hjm_surrogate_error_table",
            "hjm_surrogate_save", "hjm_surrogate_load", "hjm_surrogate_destroy", "hjm_mlp_gemm",
            "hjm_trace_enable", "hjm_trace_read", "hjm_tile_get", "hjm_tile_set", "hjm_autotune",
            "hjm_wait_status", "hjm_test_drop_plane", "hjm_price_strip", "hjm_surrogate_premium",
            "hjm_surrogate_gauss_premium", "hjm_status_string",
            "hjm_last_error")


class HJMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (hjm_status_string(status), msg))
        self.status = status


def hjm_status_string(status):
    return lib.hjm_status_string(int(status)).decode()


def hjm_last_error():
    return lib.hjm_last_error().decode()


def _check(status):
    if status != HJM_OK:
        raise HJMError(status, hjm_last_error())


# ------------------------------------------------------------- marshalling

def _struct(t, d, rename=None):
    s = t()
    for name, typ in t._fields_:
        key = (rename or {}).get(name, name)
        if hasattr(typ, "_length_"):  # fixed-size array: the given values, zero-padded
            vals = [float(v) for v in d.get(key, ())]
            if len(vals) > typ._length_:
                raise ValueError("%s holds at most %d values" % (key, typ._length_))
            getattr(s, name)[:len(vals)] = vals
        elif name == "n_knots":
            setattr(s, name, int(d.get(key, 0)))
        else:
            setattr(s, name, d[key])
    return s


def curve_struct(d):
    return _struct(hjm_curve, d)


def model_struct(d):
    return _struct(hjm_model_params, d)


def grid_struct(d):
    return _struct(hjm_grid_spec, d)


def inst_struct(d):
    return _struct(hjm_instrument, d, {"expiry_T": "T", "pay_TM": "TM", "strike_K": "K"})


def batch_item(d):
    return hjm_batch_item(curve_struct(d["curve"]), model_struct(d["model"]),
                          grid_struct(d["grid"]), inst_struct(d["inst"]))


def _ptr(x):
    """Address of a torch tensor, numpy array or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("expected a tensor, an array or an address")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- the ABI

def hjm_grid_create(curve, model, spec, stream=None):
    h = C.c_void_p()
    _check(lib.hjm_grid_create(C.byref(curve_struct(curve)), C.byref(model_struct(model)),
                               C.byref(grid_struct(spec)), _stream(stream), C.byref(h)))
    return h


def hjm_grid_destroy(handle):
    _check(lib.hjm_grid_destroy(handle))


def hjm_price(handle, inst, precision=HJM_FP32, tol_rel=1e-4, with_info=False):
    p = C.c_double()
    info = hjm_price_info()
    _check(lib.hjm_price(handle, C.byref(inst_struct(inst)), PRECISIONS[precision], float(tol_rel),
                         C.byref(p), C.byref(info) if with_info else None))
    return (p.value, info) if with_info else p.value


def make_items(items):
    arr = (hjm_batch_item * len(items))()
    for i, d in enumerate(items):
        arr[i] = batch_item(d)
    return arr


def hjm_price_batch(items, precision=HJM_FP32, tol_rel=1e-4, out=None, infos=False, stream=None):
    """items: list of item dicts or a ctypes array from make_items(). out:
    torch tensor (device or host) or numpy array of n doubles; a numpy array
    is allocated when out is None. Returns out (and infos if asked)."""
    arr = items if isinstance(items, C.Array) else make_items(items)
    n = len(arr)
    if out is None:
        out = np.empty(n, dtype=np.float64)
    inf = (hjm_price_info * n)() if infos else None
    _check(lib.hjm_price_batch(arr, n, PRECISIONS[precision], float(tol_rel), _ptr(out),
                               inf, _stream(stream)))
    return (out, inf) if infos else out


def hjm_field(handle, inst, precision, n_run, out):
    _check(lib.hjm_field(handle, C.byref(inst_struct(inst)), PRECISIONS[precision], int(n_run), _ptr(out)))
    return out


def hjm_axis(handle, inst, axis, n):
    z, J, J2 = np.empty(n), np.empty(n), np.empty(n)
    _check(lib.hjm_axis(handle, C.byref(inst_struct(inst)), int(axis), z.ctypes.data, J.ctypes.data,
                        J2.ctypes.data))
    return z, J, J2


def hjm_douglas_pass(handle, inst, precision, pass_, step_n, inp, inp2, out):
    _check(lib.hjm_douglas_pass(handle, C.byref(inst_struct(inst)), PRECISIONS[precision], int(pass_),
                                int(step_n), _ptr(inp), _ptr(inp2), _ptr(out)))
    return out


def hjm_price_static(item, precision, out, stream=None):
    """Allocation-free price of one item into out (a device tensor of one
    double); see hjm.h for the limits and the ordering rule."""
    it = item if isinstance(item, hjm_batch_item) else batch_item(item)
    _check(lib.hjm_price_static(C.byref(it), PRECISIONS[precision], _ptr(out), _stream(stream)))
    return out


def hjm_tile_get(n_r, n_v, n_y, precision=HJM_FP32):
    """Launch shape in use for a grid shape: (p1_lanes, p1_nodes, p1_lines, p2_warps, p3_warps,
    p1_staged, p1_planes)."""
    t = hjm_tile()
    _check(lib.hjm_tile_get(int(n_r), int(n_v), int(n_y), PRECISIONS[precision], C.byref(t)))
    return (t.p1_lanes, t.p1_nodes, t.p1_lines, t.p2_warps, t.p3_warps, t.p1_staged, t.p1_planes)


def hjm_tile_set(n_r, n_v, n_y, precision=HJM_FP32, tile=None):
    """Fix the launch shape of a grid shape (a 7-tuple, or 5 values with p1_staged = 0), or
    restore the default (None)."""
    vals = [int(x) for x in tile] + [0] * (7 - len(tile)) if tile is not None else None
    ptr = C.byref(hjm_tile(*vals)) if tile is not None else None
    _check(lib.hjm_tile_set(int(n_r), int(n_v), int(n_y), PRECISIONS[precision], ptr))


def hjm_autotune(items, precision=HJM_FP32, steps=8, stream=None):
    """Time every candidate launch shape on the items' grid shapes and keep the fastest."""
    arr = items if isinstance(items, C.Array) else make_items(items)
    _check(lib.hjm_autotune(arr, len(arr), PRECISIONS[precision], int(steps), _stream(stream)))


def hjm_price_strip(items, precision=HJM_FP32, tol_rel=1e-4, stream=None):
    """A cap or floor from its strip of caplets / floorlets: (total, per period)."""
    arr = items if isinstance(items, C.Array) else make_items(items)
    total = C.c_double()
    each = (C.c_double * len(arr))()
    _check(lib.hjm_price_strip(arr, len(arr), PRECISIONS[precision], float(tol_rel), C.byref(total), each,
                               _stream(stream)))
    return float(total.value), [float(v) for v in each]


def hjm_wait_status(reset=False):
    """Raises HJMError (HJM_ETIMEOUT) when a bounded device wait gave up."""
    _check(lib.hjm_wait_status(1 if reset else 0))


def hjm_test_drop_plane(plane, polls=0):
    """Test hook: y plane `plane` is never copied by the TMA-fed pass 1 (-1: off)."""
    _check(lib.hjm_test_drop_plane(int(plane), int(polls)))


def hjm_trace_enable(on):
    _check(lib.hjm_trace_enable(1 if on else 0))


def hjm_trace_read(reset=False):
    """Per-kind launch counts and total device ms, as a dict."""
    t = hjm_trace()
    _check(lib.hjm_trace_read(C.byref(t), 1 if reset else 0))
    return {name: (int(t.launches[i]), float(t.total_ms[i])) for i, name in enumerate(TRACE_KIND_NAMES)}


# ---------------------------------------------------------------- surrogate

def surrogate_cfg(n_train, epochs, batch, lr, seed, box_lo, box_hi, label_grid, checkpoint_path=None):
    c = hjm_surrogate_cfg()
    c.n_train = int(n_train)
    c.hidden, c.depth = 256, 4
    c.epochs, c.batch, c.lr, c.seed = int(epochs), int(batch), float(lr), int(seed)
    for k in range(9):
        c.box_lo[k] = float(box_lo[k])
        c.box_hi[k] = float(box_hi[k])
    c.label_grid = grid_struct(label_grid)
    c.checkpoint_path = checkpoint_path.encode() if checkpoint_path else None
    return c


def hjm_surrogate_create(cfg, stream=None):
    h = C.c_void_p()
    _check(lib.hjm_surrogate_create(C.byref(cfg), _stream(stream), C.byref(h)))
    return h


def hjm_surrogate_train(cfg, stream=None):
    h = C.c_void_p()
    _check(lib.hjm_surrogate_train(C.byref(cfg), _stream(stream), C.byref(h)))
    return h


def hjm_surrogate_fit(h, x, t, epochs, stream=None):
    loss = C.c_float()
    n = int(t.numel() if hasattr(t, "numel") else len(t))
    _check(lib.hjm_surrogate_fit(h, _ptr(x), _ptr(t), n, int(epochs), _stream(stream), C.byref(loss)))
    return loss.value


def hjm_surrogate_infer(h, x, price_out, used_pde=None, stream=None):
    n = int(price_out.numel() if hasattr(price_out, "numel") else len(price_out))
    _check(lib.hjm_surrogate_infer(h, _ptr(x), n, _ptr(price_out), _ptr(used_pde), _stream(stream)))
    return price_out


def hjm_surrogate_forward(h, x, y_out, stream=None):
    n = int(y_out.numel() if hasattr(y_out, "numel") else len(y_out))
    _check(lib.hjm_surrogate_forward(h, _ptr(x), n, _ptr(y_out), _stream(stream)))
    return y_out


def hjm_surrogate_premium(h, x, premium_out, stream=None):
    """The network alone as forward premia (Gaussian part + learned correction)."""
    n = int(premium_out.numel() if hasattr(premium_out, "numel") else len(premium_out))
    _check(lib.hjm_surrogate_premium(h, _ptr(x), n, _ptr(premium_out), _stream(stream)))
    return premium_out


def hjm_surrogate_gauss_premium(x, premium_out, stream=None):
    """The closed-form Gaussian-HJM forward premium of each row."""
    n = int(premium_out.numel() if hasattr(premium_out, "numel") else len(premium_out))
    _check(lib.hjm_surrogate_gauss_premium(_ptr(x), n, _ptr(premium_out), _stream(stream)))
    return premium_out


def hjm_surrogate_loss_grad(h, x, t, grad_out, stream=None):
    loss = C.c_float()
    n = int(t.numel() if hasattr(t, "numel") else len(t))
    _check(lib.hjm_surrogate_loss_grad(h, _ptr(x), _ptr(t), n, C.byref(loss), _ptr(grad_out), _stream(stream)))
    return loss.value


def hjm_surrogate_get_params(h):
    out = np.empty(HJM_SURROGATE_PARAMS, dtype=np.float32)
    _check(lib.hjm_surrogate_get_params(h, out.ctypes.data))
    return out


def hjm_surrogate_set_params(h, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == HJM_SURROGATE_PARAMS
    _check(lib.hjm_surrogate_set_params(h, p.ctypes.data))


def hjm_surrogate_error_table(h):
    out = np.empty(HJM_SURROGATE_BINS, dtype=np.float32)
    _check(lib.hjm_surrogate_error_table(h, out.ctypes.data))
    return out


def hjm_surrogate_save(h, path):
    _check(lib.hjm_surrogate_save(h, path.encode()))


def hjm_surrogate_load(path):
    h = C.c_void_p()
    _check(lib.hjm_surrogate_load(path.encode(), C.byref(h)))
    return h


def hjm_surrogate_destroy(h):
    _check(lib.hjm_surrogate_destroy(h))


def hjm_mlp_gemm(M, N, K, A, lda, trans_a, B, ldb, trans_b, C_out, ldc, stream=None):
    _check(lib.hjm_mlp_gemm(int(M), int(N), int(K), _ptr(A), int(lda), int(bool(trans_a)), _ptr(B), int(ldb),
                            int(bool(trans_b)), _ptr(C_out), int(ldc), _stream(stream)))
    return C_out


class Grid:
    """Owning wrapper of an hjm_grid handle built from an item dict."""

    def __init__(self, item, stream=None):
        self.item = item
        self.h = hjm_grid_create(item["curve"], item["model"], item["grid"], stream)
        g = item["grid"]
        self.shape = (g["n_y"], g["n_v"], g["n_r"])

    def close(self):
        if getattr(self, "h", None) is not None:
            hjm_grid_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    __del__ = close

    def price(self, precision=HJM_FP32, inst=None, with_info=False):
        return hjm_price(self.h, inst or self.item["inst"], precision, with_info=with_info)

    def field(self, precision, n_run, out):
        return hjm_field(self.h, self.item["inst"], precision, n_run, out)

    def axis(self, axis):
        return hjm_axis(self.h, self.item["inst"], axis, self.shape[2 - axis])

    def douglas_pass(self, precision, pass_, step_n, inp, inp2, out):
        return hjm_douglas_pass(self.h, self.item["inst"], precision, pass_, step_n, inp, inp2, out)
