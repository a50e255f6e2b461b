"""Thin ctypes binding of libphpp.so (include/phpp.h), same names as the C ABI.

Only argument marshalling lives here: tensors become raw pointers, the
current torch CUDA stream becomes the cudaStream_t, return codes become
exceptions.  Every step of the computation runs in the library's kernels.
If the library is missing, every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import warnings
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PHPP_LIB selects another build of the same library (e.g. the bounds-checked
# libphpp_checked.so); the default is the normal build.
LIB_PATH = os.environ.get("PHPP_LIB") or os.path.join(_HERE, "libphpp.so")

PH_OK = 0
PH_WARN_FALLBACK = 1
PH_ERR_ARG = -1
PH_ERR_RCUT_GE_HALF_L = -2
PH_ERR_NONFINITE = -3
PH_ERR_OOM = -4
PH_ERR_CUDA = -5
PH_ERR_CAPACITY = -6
PH_ERR_TIMEOUT = -7
PH_ERR_STATE = -8
PH_F32, PH_F64 = 0, 1
PH_KEY_MORTON, PH_KEY_HILBERT = 0, 1
PH_G_EXACT, PH_G_LEARNED, PH_G_TABLE = 0, 1, 2


class PhError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"phpp error {code}: {msg}")
        self.code = code


class ph_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("G", ctypes.c_double), ("eps", ctypes.c_double),
                ("rs", ctypes.c_double), ("rcut", ctypes.c_double), ("leaf_max", ctypes.c_int32),
                ("key_kind", ctypes.c_int32), ("group_size", ctypes.c_int32), ("level_bits", ctypes.c_int32),
                ("pp_variant", ctypes.c_int32), ("queue_order", ctypes.c_int32), ("theta", ctypes.c_double)]


class ph_leaves_view(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_boxes", ctypes.c_int32), ("n_leaves", ctypes.c_int32),
                ("n_groups", ctypes.c_int32), ("n_cells", ctypes.c_int32),
                ("keys", ctypes.c_void_p), ("perm", ctypes.c_void_p), ("leaf_first", ctypes.c_void_p),
                ("leaf_ref", ctypes.c_void_p), ("leaf_half", ctypes.c_void_p),
                ("group_first", ctypes.c_void_p), ("group_ref", ctypes.c_void_p),
                ("group_half", ctypes.c_void_p), ("pos_leaf", ctypes.c_void_p),
                ("pos_group", ctypes.c_void_p), ("cell_leaf_first", ctypes.c_void_p),
                ("g", ctypes.c_int32 * 4), ("key_bits", ctypes.c_int32), ("group_size", ctypes.c_int32)]


class ph_train_params(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int64), ("batch", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("lr0", ctypes.c_float), ("lr_min", ctypes.c_float), ("tol", ctypes.c_float),
                ("reserved", ctypes.c_int32), ("seed", ctypes.c_uint64)]


PH_MLP_PARAMS = 321
PH_TUNE_MAX = 32


class ph_tune_result(ctypes.Structure):
    _fields_ = [("best", ph_params), ("best_ms", ctypes.c_float), ("n_tried", ctypes.c_int32),
                ("ms", ctypes.c_float * PH_TUNE_MAX), ("leaf_max", ctypes.c_int32 * PH_TUNE_MAX),
                ("level_bits", ctypes.c_int32 * PH_TUNE_MAX), ("pp_variant", ctypes.c_int32 * PH_TUNE_MAX),
                ("group_size", ctypes.c_int32 * PH_TUNE_MAX), ("key_kind", ctypes.c_int32 * PH_TUNE_MAX)]


class ph_pairs_view(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int64), ("n_groups", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("group_off", ctypes.c_void_p), ("entries", ctypes.c_void_p), ("counts", ctypes.c_void_p),
                ("group_order", ctypes.c_void_p)]


class ph_pm_view(ctypes.Structure):
    _fields_ = [("n_mesh", ctypes.c_int32), ("reserved", ctypes.c_int32), ("mass_unit", ctypes.c_double),
                ("mass_fixed", ctypes.c_void_p), ("mesh", ctypes.c_void_p)]


PH_PM_MAX_MESH = 1024
PH_CLOCK_NEWTON, PH_CLOCK_LCDM = 0, 1


class ph_kdk_params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("eta", ctypes.c_double), ("eps_step", ctypes.c_double),
                ("H0", ctypes.c_double), ("omega_m", ctypes.c_double), ("omega_l", ctypes.c_double),
                ("max_level", ctypes.c_int32), ("n_mesh", ctypes.c_int32), ("clock", ctypes.c_int32),
                ("g_mode", ctypes.c_int32)]

_lib = None

_VP = ctypes.c_void_p
_SIGS = {
    "ph_build_leaves": ([_VP, ctypes.c_int, _VP, ctypes.c_int64, ctypes.POINTER(ph_params), _VP,
                         ctypes.POINTER(_VP)], ctypes.c_int),
    "ph_build_leaves_batched": ([_VP, ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                 ctypes.POINTER(ph_params), _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "ph_leaf_pairs": ([_VP, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "ph_pairs_reserve": ([ctypes.POINTER(_VP), ctypes.c_int64], ctypes.c_int),
    "ph_pp_accel": ([_VP, _VP, ctypes.c_int, _VP, _VP, _VP], ctypes.c_int),
    "ph_accel": ([_VP, ctypes.c_int, _VP, ctypes.c_int64, ctypes.POINTER(ph_params), ctypes.c_int, _VP, _VP, _VP,
                  ctypes.POINTER(_VP), ctypes.POINTER(_VP)], ctypes.c_int),
    "ph_free": ([_VP], None),
    "ph_last_error": ([], ctypes.c_char_p),
    "ph_status": ([_VP], ctypes.c_int),
    "ph_leaves_get_view": ([_VP, ctypes.POINTER(ph_leaves_view)], ctypes.c_int),
    "ph_pairs_get_view": ([_VP, ctypes.POINTER(ph_pairs_view)], ctypes.c_int),
    "ph_pp_counters": ([_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "ph_count_within": ([_VP, _VP, ctypes.POINTER(ctypes.c_int64), _VP], ctypes.c_int),
    "ph_launch_counter": ([], ctypes.c_int64),
    "ph_accel_noalloc": ([_VP, _VP, ctypes.c_int64, ctypes.POINTER(ph_params), _VP, _VP], ctypes.c_int),
    "ph_mlp_train": ([ctypes.POINTER(ph_train_params), ctypes.c_double, ctypes.c_double, _VP, _VP,
                      ctypes.POINTER(_VP)], ctypes.c_int),
    "ph_mlp_create": ([_VP, ctypes.c_double, ctypes.c_double, ctypes.c_float, _VP, ctypes.POINTER(_VP)],
                      ctypes.c_int),
    "ph_mlp_get": ([_VP, _VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "ph_mlp_loss_grad": ([_VP, _VP, _VP, ctypes.c_int64, _VP, ctypes.POINTER(ctypes.c_float), _VP], ctypes.c_int),
    "ph_mlp_file_write": ([ctypes.c_char_p, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_float, ctypes.c_float,
                           ctypes.c_int32], ctypes.c_int),
    "ph_mlp_file_read": ([ctypes.c_char_p, _VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                          ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "ph_mlp_save": ([_VP, ctypes.c_char_p], ctypes.c_int),
    "ph_mlp_load": ([ctypes.c_char_p, ctypes.c_float, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "ph_debug_fail_allocation": ([ctypes.c_int64], None),
    "ph_mlp_eval": ([_VP, _VP, ctypes.c_int64, _VP, _VP], ctypes.c_int),
    "ph_debug_bounds": ([ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "ph_graph_create": ([_VP, _VP, _VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP, ctypes.c_double, _VP,
                         ctypes.POINTER(_VP)], ctypes.c_int),
    "ph_graph_launch": ([_VP, _VP], ctypes.c_int),
    "ph_graph_launch_host": ([_VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "ph_graph_launch_host_async": ([_VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "ph_graph_kernels": ([_VP, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "ph_pm_accel": ([_VP, ctypes.c_int, _VP, ctypes.c_int64, ctypes.POINTER(ph_params), ctypes.c_int32, _VP, _VP,
                     ctypes.c_int32, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "ph_pm_get_view": ([_VP, ctypes.POINTER(ph_pm_view)], ctypes.c_int),
    "ph_sim_create": ([_VP, _VP, _VP, ctypes.c_int64, ctypes.POINTER(ph_params), ctypes.POINTER(ph_kdk_params),
                       ctypes.c_double, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "ph_sim_step": ([_VP, ctypes.c_int32, _VP], ctypes.c_int),
    "ph_sim_get": ([_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)],
                   ctypes.c_int),
    "ph_domain_cells": ([_VP, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ph_params), ctypes.POINTER(ctypes.c_int32),
                         _VP], ctypes.c_int),
    "ph_domain_partition": ([_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP, _VP], ctypes.c_int),
    "ph_domain_halo": ([_VP, ctypes.c_int32, ctypes.c_int32, _VP], ctypes.c_int),
    "ph_leaves_set_active": ([_VP, _VP, ctypes.c_int64], ctypes.c_int),
    "ph_domain_cells_device": ([_VP, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ph_params),
                                ctypes.POINTER(ctypes.c_int32), _VP, _VP, _VP], ctypes.c_int),
    "ph_domain_pack": ([_VP, ctypes.c_int, _VP, _VP, _VP, ctypes.c_int64, _VP, ctypes.c_int32, ctypes.c_int32, _VP,
                        ctypes.c_int64, _VP, _VP], ctypes.c_int),
    "ph_domain_unpack": ([_VP, ctypes.c_int64, ctypes.c_int, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_int64), _VP],
                         ctypes.c_int),
    "ph_autotune": ([_VP, ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, ctypes.POINTER(ph_params),
                     ctypes.c_int32, _VP, ctypes.POINTER(ph_tune_result)], ctypes.c_int),
}


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc):
    if rc < 0:
        raise PhError(rc, lib().ph_last_error().decode())
    if rc > 0:
        warnings.warn(f"phpp warning {rc}: {lib().ph_last_error().decode()}")
    return rc


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return ctypes.c_void_p(t.ctypes.data)
    assert t.is_contiguous(), "tensors must be contiguous"
    return ctypes.c_void_p(t.data_ptr())


def _pos_type(t):
    import torch
    dt = t.dtype
    if dt in (np.float32, torch.float32):
        return PH_F32
    if dt in (np.float64, torch.float64):
        return PH_F64
    raise TypeError("positions must be float32 or float64")


def make_params(L, G, eps, rs, rcut, leaf_max=32, key_kind=PH_KEY_MORTON, group_size=0, level_bits=0,
                pp_variant=0, theta=0.0, queue_order=0):
    return ph_params(float(L), float(G), float(eps), float(rs), float(rcut), int(leaf_max), int(key_kind),
                     int(group_size), int(level_bits), int(pp_variant), int(queue_order), float(theta))


class Handle:
    """Owner of a ph_leaves / ph_pairs handle (freed on close or collection)."""

    def __init__(self, ptr, keep=()):
        self.ptr = ctypes.c_void_p(ptr)
        self._keep = keep
        self._fin = weakref.finalize(self, _free_ptr, ptr)

    def close(self):
        self._fin()

    @property
    def as_arg(self):
        return self.ptr


def _free_ptr(p):
    if _lib is not None and p:
        _lib.ph_free(ctypes.c_void_p(p))


def _handle_in(h):
    return ctypes.c_void_p(h.ptr.value if h is not None else None)


def _wrap(out, h, keep=()):
    if h is not None and h.ptr.value == out.value:
        h._keep = keep
        return h
    return Handle(out.value, keep)


def ph_build_leaves(pos, mass, params, stream=None, leaves=None):
    """Sort particles into leaves and target groups (host or device tensors)."""
    out = _handle_in(leaves)
    n = int(pos.shape[0])
    _check(lib().ph_build_leaves(_ptr(pos), _pos_type(pos), _ptr(mass), n, ctypes.byref(params),
                                 _stream(stream), ctypes.byref(out)))
    return _wrap(out, leaves, (pos, mass))


def ph_build_leaves_batched(pos, mass, box_offsets, params_list, stream=None, leaves=None):
    out = _handle_in(leaves)
    offs = np.ascontiguousarray(np.asarray(box_offsets, np.int64))
    nb = offs.size - 1
    arr = (ph_params * nb)(*params_list)
    _check(lib().ph_build_leaves_batched(_ptr(pos), _pos_type(pos), _ptr(mass),
                                         offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), nb, arr,
                                         _stream(stream), ctypes.byref(out)))
    return _wrap(out, leaves, (pos, mass, offs, arr))


def ph_leaf_pairs(leaves, stream=None, pairs=None):
    out = _handle_in(pairs)
    _check(lib().ph_leaf_pairs(leaves.ptr, _stream(stream), ctypes.byref(out)))
    return _wrap(out, pairs)


def ph_pairs_reserve(capacity, pairs=None):
    out = _handle_in(pairs)
    _check(lib().ph_pairs_reserve(ctypes.byref(out), int(capacity)))
    return _wrap(out, pairs)


def ph_pp_accel(leaves, pairs, g_mode, mlp, acc, stream=None):
    """Accelerations into ``acc`` [N,3] float32 (host or device), caller order.
    pairs = None: the direct mode (leaf pairs found in the kernel)."""
    return _check(lib().ph_pp_accel(leaves.ptr, pairs.ptr if pairs is not None else None, int(g_mode),
                                    mlp.ptr if mlp is not None else None, _ptr(acc), _stream(stream)))


def ph_accel(pos, mass, params, g_mode, mlp, acc, stream=None, leaves=None, pairs=None, direct=False):
    """Whole step: build, pairs, PP.  Returns (leaves, pairs) handles for reuse.
    direct=True: build and the direct-mode PP, no pair list (pairs is None)."""
    lo = _handle_in(leaves)
    po = _handle_in(pairs)
    rc = lib().ph_accel(_ptr(pos), _pos_type(pos), _ptr(mass), int(pos.shape[0]), ctypes.byref(params), int(g_mode),
                        mlp.ptr if mlp is not None else None, _ptr(acc), _stream(stream), ctypes.byref(lo),
                        None if direct else ctypes.byref(po))
    lh = _wrap(lo, leaves, (pos, mass)) if lo.value else None
    ph = _wrap(po, pairs) if (po.value and not direct) else None
    _check(rc)
    return lh, ph


def ph_free(handle):
    if handle is not None:
        handle.close()


def ph_status(handle):
    return _check(lib().ph_status(handle.ptr))


def ph_last_error():
    return lib().ph_last_error().decode()


def ph_pp_counters(handle):
    """(interactions evaluated, sources staged) of the last PP call: the pairs
    handle it used, or its leaves handle after a direct-mode call."""
    a = ctypes.c_int64(0)
    b = ctypes.c_int64(0)
    _check(lib().ph_pp_counters(handle.ptr, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def ph_count_within(leaves, pairs, stream=None):
    """Ordered pairs j != i with r < rcut in the lists (synchronises)."""
    n = ctypes.c_int64(0)
    _check(lib().ph_count_within(leaves.ptr, pairs.ptr, ctypes.byref(n), _stream(stream)))
    return n.value


def ph_accel_noalloc(pos, mass, params, acc, stream=None):
    """Whole exact-factor step for one small box using only the library's
    fixed scratch array (no device allocation); device tensors only."""
    return _check(lib().ph_accel_noalloc(_ptr(pos), _ptr(mass), int(pos.shape[0]), ctypes.byref(params),
                                         _ptr(acc), _stream(stream)))


def make_train_params(n_samples=1_000_000, batch=4096, steps=40_000, lr0=1e-2, lr_min=1e-5, tol=1e-3, seed=12345):
    return ph_train_params(int(n_samples), int(batch), int(steps), float(lr0), float(lr_min), float(tol), 0,
                           int(seed))


def ph_mlp_train(tp, rs, rcut, init_weights=None, stream=None):
    """Train the 1-16-16-1 network on the GPU; returns the handle."""
    out = ctypes.c_void_p(None)
    w = None if init_weights is None else np.ascontiguousarray(np.asarray(init_weights, np.float32))
    _check(lib().ph_mlp_train(ctypes.byref(tp), float(rs), float(rcut), _ptr(w), _stream(stream),
                              ctypes.byref(out)))
    return Handle(out.value)


def ph_mlp_create(weights, rs, rcut, tol=0.0, stream=None):
    out = ctypes.c_void_p(None)
    w = np.ascontiguousarray(np.asarray(weights, np.float32))
    _check(lib().ph_mlp_create(_ptr(w), float(rs), float(rcut), float(tol), _stream(stream), ctypes.byref(out)))
    return Handle(out.value)


def ph_mlp_eval(mlp, z0, out, stream=None):
    """g_hat at the inputs z0 (device float32 tensor) into out, as the
    learned PP kernel evaluates it."""
    return _check(lib().ph_mlp_eval(mlp.ptr, _ptr(z0), int(z0.numel()), _ptr(out), _stream(stream)))


def ph_mlp_get(mlp):
    """(weights float32[321], validated max relative error, last loss)."""
    w = np.zeros(PH_MLP_PARAMS, np.float32)
    e = ctypes.c_float(0)
    l = ctypes.c_float(0)
    _check(lib().ph_mlp_get(mlp.ptr, _ptr(w), ctypes.byref(e), ctypes.byref(l)))
    return w, e.value, l.value


def ph_mlp_file_write(path, weights, rs, rcut, max_rel_err=0.0, last_loss=0.0, steps=0):
    """Write a network file (host only; layout in phpp.h)."""
    w = np.ascontiguousarray(np.asarray(weights, np.float32))
    assert w.size == PH_MLP_PARAMS
    _check(lib().ph_mlp_file_write(os.fsencode(path), _ptr(w), float(rs), float(rcut), float(max_rel_err),
                                   float(last_loss), int(steps)))


def ph_mlp_file_read(path):
    """(weights float32[321], rs, rcut, max_rel_err, last_loss, steps) of a network file (host only)."""
    w = np.zeros(PH_MLP_PARAMS, np.float32)
    rs, rcut = ctypes.c_double(0), ctypes.c_double(0)
    err, loss = ctypes.c_float(0), ctypes.c_float(0)
    steps = ctypes.c_int32(0)
    _check(lib().ph_mlp_file_read(os.fsencode(path), _ptr(w), ctypes.byref(rs), ctypes.byref(rcut), ctypes.byref(err),
                                  ctypes.byref(loss), ctypes.byref(steps)))
    return w, rs.value, rcut.value, err.value, loss.value, steps.value


def ph_mlp_save(mlp, path):
    _check(lib().ph_mlp_save(mlp.ptr, os.fsencode(path)))


def ph_mlp_load(path, tol=0.0, stream=None):
    out = ctypes.c_void_p(None)
    _check(lib().ph_mlp_load(os.fsencode(path), float(tol), _stream(stream), ctypes.byref(out)))
    return Handle(out.value)


def ph_debug_fail_allocation(k):
    """Make the k-th next device allocation of the library fail (k < 0: off)."""
    lib().ph_debug_fail_allocation(int(k))


def ph_debug_bounds():
    """(out-of-bounds accesses skipped since the last call, site of the first)
    of a library built with bounds checks; raises from a normal build."""
    h = ctypes.c_int64(0)
    s = ctypes.c_int32(0)
    _check(lib().ph_debug_bounds(ctypes.byref(h), ctypes.byref(s)))
    return h.value, s.value


def ph_mlp_loss_grad(weights, z0, target, stream=None):
    """Gradient (float32[321]) and loss of one forward/backward pass."""
    w = np.ascontiguousarray(np.asarray(weights, np.float32))
    z = np.ascontiguousarray(np.asarray(z0, np.float32))
    t = np.ascontiguousarray(np.asarray(target, np.float32))
    g = np.zeros(PH_MLP_PARAMS, np.float32)
    loss = ctypes.c_float(0)
    _check(lib().ph_mlp_loss_grad(_ptr(w), _ptr(z), _ptr(t), int(z.size), _ptr(g), ctypes.byref(loss),
                                  _stream(stream)))
    return g, loss.value


def ph_graph_create(leaves, pairs, pos, mass, g_mode, mlp, acc, headroom=0.25, stream=None):
    """Capture build + pairs + PP for these handles as one CUDA graph."""
    out = ctypes.c_void_p(None)
    _check(lib().ph_graph_create(leaves.ptr, pairs.ptr if pairs is not None else None, _ptr(pos), _pos_type(pos),
                                 _ptr(mass), int(g_mode),
                                 mlp.ptr if mlp is not None else None, _ptr(acc), float(headroom), _stream(stream),
                                 ctypes.byref(out)))
    return Handle(out.value, (leaves, pairs, pos, mass, acc, mlp))


def ph_graph_launch(graph, stream=None):
    return _check(lib().ph_graph_launch(graph.ptr, _stream(stream)))


def ph_graph_launch_host(graph, pos, mass, acc, stream=None):
    """Copy host pos/mass in, replay, copy acc out (synchronises)."""
    return _check(lib().ph_graph_launch_host(graph.ptr, _ptr(pos), _ptr(mass), _ptr(acc), _stream(stream)))


def ph_graph_launch_host_async(graph, pos, mass, acc, stream=None):
    """Enqueue the copies in, the replay and the copy out without waiting;
    acc is valid after the stream is synchronised (pinned host tensors)."""
    return _check(lib().ph_graph_launch_host_async(graph.ptr, _ptr(pos), _ptr(mass), _ptr(acc), _stream(stream)))


def ph_graph_kernels(graph):
    k = ctypes.c_int64(0)
    _check(lib().ph_graph_kernels(graph.ptr, ctypes.byref(k)))
    return k.value


def ph_autotune(pos, mass, box_offsets, params_list, reps=3, stream=None):
    """Time every tuner candidate on these particles; returns ph_tune_result."""
    offs = np.ascontiguousarray(np.asarray(box_offsets, np.int64))
    nb = offs.size - 1
    arr = (ph_params * nb)(*params_list)
    res = ph_tune_result()
    _check(lib().ph_autotune(_ptr(pos), _pos_type(pos), _ptr(mass), offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             nb, arr, int(reps), _stream(stream), ctypes.byref(res)))
    return res


def ph_pm_accel(pos, mass, params, n_mesh, acc, pot=None, accumulate=False, stream=None, pm=None):
    """Long-range PM acceleration into ``acc`` [N,3] (added to it when
    ``accumulate``), optional potential into ``pot`` [N]; host or device
    tensors.  Returns the ph_pm handle for reuse."""
    out = _handle_in(pm)
    rc = lib().ph_pm_accel(_ptr(pos), _pos_type(pos), _ptr(mass), int(pos.shape[0]), ctypes.byref(params),
                           int(n_mesh), _ptr(acc), _ptr(pot), int(bool(accumulate)), _stream(stream),
                           ctypes.byref(out))
    h = _wrap(out, pm) if out.value else None
    _check(rc)
    return h


def ph_pm_get_view(pm):
    """Device views: fixed-point node masses (int64 [N,N,N]) with their unit,
    and the per-node (-grad phi, phi) mesh (float32 [N,N,N,4])."""
    v = ph_pm_view()
    _check(lib().ph_pm_get_view(pm.ptr, ctypes.byref(v)))
    n = v.n_mesh
    return {"n_mesh": n, "mass_unit": v.mass_unit,
            "mass_fixed": _dev(v.mass_fixed, (n, n, n), "<i8"),
            "mesh": _dev(v.mesh, (n, n, n, 4), "<f4")}


def make_kdk_params(dt, eta, max_level, n_mesh=0, eps_step=0.0, clock=PH_CLOCK_NEWTON, H0=1.0, omega_m=1.0,
                    omega_l=0.0, g_mode=PH_G_EXACT):
    return ph_kdk_params(float(dt), float(eta), float(eps_step), float(H0), float(omega_m), float(omega_l),
                         int(max_level), int(n_mesh), int(clock), int(g_mode))


def ph_sim_create(pos, mom, mass, params, kp, t0=0.0, stream=None):
    """New simulation from float64 positions/momenta [N,3] and float32 masses
    (host or device tensors / arrays; mass None = 1/N)."""
    out = ctypes.c_void_p(None)
    _check(lib().ph_sim_create(_ptr(pos), _ptr(mom), _ptr(mass), int(pos.shape[0]), ctypes.byref(params),
                               ctypes.byref(kp), float(t0), _stream(stream), ctypes.byref(out)))
    return Handle(out.value)


def ph_sim_step(sim, n_steps=1, stream=None):
    return _check(lib().ph_sim_step(sim.ptr, int(n_steps), _stream(stream)))


def ph_sim_get(sim, n):
    """(positions float64 [N,3], momenta float64 [N,3], accelerations float32
    [N,3], levels int32 [N], time, force passes) as numpy arrays."""
    x = np.zeros((n, 3))
    p = np.zeros((n, 3))
    a = np.zeros((n, 3), np.float32)
    lv = np.zeros(n, np.int32)
    t = ctypes.c_double(0)
    fp = ctypes.c_int64(0)
    _check(lib().ph_sim_get(sim.ptr, _ptr(x), _ptr(p), _ptr(a), _ptr(lv), ctypes.byref(t), ctypes.byref(fp)))
    return x, p, a, lv, t.value, fp.value


def ph_domain_cells(pos, params):
    """(N_side, ground cell of every particle) for host positions [N,3]
    (numpy or CPU tensor, float32 or float64); runs on the host."""
    a = np.ascontiguousarray(pos.numpy() if hasattr(pos, "numpy") else pos)
    cells = np.zeros(a.shape[0], np.int32)
    ns = ctypes.c_int32(0)
    _check(lib().ph_domain_cells(_ptr(a), _pos_type(a), int(a.shape[0]), ctypes.byref(params), ctypes.byref(ns),
                                 _ptr(cells)))
    return ns.value, cells


def ph_domain_partition(cell_count, nside, key_kind, n_domains):
    """(owner int32 [N_side^3], work per domain float64 [n_domains])."""
    c = np.ascontiguousarray(np.asarray(cell_count, np.int64))
    owner = np.zeros(c.size, np.int32)
    cost = np.zeros(int(n_domains), np.float64)
    _check(lib().ph_domain_partition(_ptr(c), int(nside), int(key_kind), int(n_domains), _ptr(owner), _ptr(cost)))
    return owner, cost


def ph_domain_halo(owner, nside, domain):
    """need uint8 [N_side^3]: 1 own cell, 2 ghost cell, 0 not needed."""
    o = np.ascontiguousarray(np.asarray(owner, np.int32))
    need = np.zeros(o.size, np.uint8)
    _check(lib().ph_domain_halo(_ptr(o), int(nside), int(domain), _ptr(need)))
    return need


PH_DOMAIN_ROW = 6


def ph_leaves_set_active(leaves, active=None):
    """Active-particle mode: ``active`` a device uint8 tensor [n] (nonzero =
    active) read at every later build of ``leaves``; None turns it off."""
    if active is None:
        _check(lib().ph_leaves_set_active(leaves.ptr, None, 0))
        leaves._active = None
        return
    assert active.dtype == __import__("torch").uint8 and active.is_cuda
    _check(lib().ph_leaves_set_active(leaves.ptr, _ptr(active), int(active.numel())))
    leaves._active = active        # kept alive with the handle


def ph_domain_cells_device(pos, params, stream=None):
    """(N_side, cell int32 [n], counts int64 [N_side^3]) on the device."""
    import torch
    n = int(pos.shape[0])
    cells = torch.empty(max(n, 1), dtype=torch.int32, device=pos.device)
    g = 0
    while g < 7 and params.L / 2.0 ** (g + 1) >= params.rcut:
        g += 1
    counts = torch.empty(8 ** g, dtype=torch.int64, device=pos.device)
    ns = ctypes.c_int32(0)
    _check(lib().ph_domain_cells_device(_ptr(pos), _pos_type(pos), n, ctypes.byref(params), ctypes.byref(ns),
                                        _ptr(cells), _ptr(counts), _stream(stream)))
    assert ns.value ** 3 == counts.numel()
    return ns.value, cells[:n], counts


def ph_domain_pack(pos, mass, ids, cells, owner, nside, n_ranks, send=None, stream=None):
    """Rows for every destination rank (device float64 [rows, PH_DOMAIN_ROW]),
    grouped by rank; returns (send buffer, rows per rank).  The buffer is
    grown (and the packing repeated) when it is too small."""
    import torch
    n = int(pos.shape[0])
    own = np.ascontiguousarray(np.asarray(owner, np.int32))
    counts = np.zeros(int(n_ranks), np.int64)
    if send is None:
        send = torch.empty((max(2 * n, 1), PH_DOMAIN_ROW), dtype=torch.float64, device=pos.device)
    rc = lib().ph_domain_pack(_ptr(pos), _pos_type(pos), _ptr(mass), _ptr(ids), _ptr(cells), n, _ptr(own), int(nside),
                              int(n_ranks), _ptr(send), int(send.shape[0]), _ptr(counts), _stream(stream))
    if rc == PH_ERR_CAPACITY:
        send = torch.empty((int(counts.sum()) + 1024, PH_DOMAIN_ROW), dtype=torch.float64, device=pos.device)
        rc = lib().ph_domain_pack(_ptr(pos), _pos_type(pos), _ptr(mass), _ptr(ids), _ptr(cells), n, _ptr(own),
                                  int(nside), int(n_ranks), _ptr(send), int(send.shape[0]), _ptr(counts),
                                  _stream(stream))
    _check(rc)
    return send, [int(c) for c in counts]


def ph_domain_unpack(recv, n_recv, pos_dtype, stream=None):
    """(pos [n_recv,3] of pos_dtype, mass float32, ids int64, n_own) of a local
    set from n_recv received rows (own particles first)."""
    import torch
    dev = recv.device
    pos = torch.empty((max(n_recv, 1), 3), dtype=pos_dtype, device=dev)
    mass = torch.empty(max(n_recv, 1), dtype=torch.float32, device=dev)
    ids = torch.empty(max(n_recv, 1), dtype=torch.int64, device=dev)
    n_own = ctypes.c_int64(0)
    _check(lib().ph_domain_unpack(_ptr(recv), int(n_recv), _pos_type(pos), _ptr(pos), _ptr(mass), _ptr(ids),
                                  ctypes.byref(n_own), _stream(stream)))
    return pos[:n_recv], mass[:n_recv], ids[:n_recv], n_own.value


def ph_launch_counter():
    return int(lib().ph_launch_counter())


# ------------------------------------------------------------ introspection
class _CudaArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2, "strides": None}


def _dev(ptr, shape, typestr):
    import torch
    if int(np.prod(shape)) == 0 or not ptr:
        dt = {"<u8": torch.int64, "<i4": torch.int32, "<f8": torch.float64, "<f4": torch.float32,
              "<i8": torch.int64, "|u1": torch.uint8}[typestr]
        return torch.zeros(shape, dtype=dt, device="cuda")
    return torch.as_tensor(_CudaArray(ptr, shape, typestr), device="cuda")


def ph_leaves_get_view(leaves):
    """Device views (torch tensors, no copy) of the handle's internal arrays."""
    v = ph_leaves_view()
    _check(lib().ph_leaves_get_view(leaves.ptr, ctypes.byref(v)))
    n, nl, ng, nc = v.n, v.n_leaves, v.n_groups, v.n_cells
    return {
        "n": n, "n_leaves": nl, "n_groups": ng, "n_cells": nc, "n_boxes": v.n_boxes,
        "g": list(v.g), "key_bits": v.key_bits, "group_size": v.group_size,
        "keys": _dev(v.keys, (n,), "<u8"),
        "perm": _dev(v.perm, (n,), "<i4"),
        "leaf_first": _dev(v.leaf_first, (nl + 1,), "<i4"),
        "leaf_ref": _dev(v.leaf_ref, (nl, 3), "<f8"),
        "leaf_half": _dev(v.leaf_half, (nl, 4), "<f4"),
        "group_first": _dev(v.group_first, (ng + 1,), "<i4"),
        "group_ref": _dev(v.group_ref, (ng, 3), "<f8"),
        "group_half": _dev(v.group_half, (ng, 4), "<f4"),
        "pos_leaf": _dev(v.pos_leaf, (n, 4), "<f4"),
        "pos_group": _dev(v.pos_group, (n, 4), "<f4"),
        "cell_leaf_first": _dev(v.cell_leaf_first, (nc + 1,), "<i4"),
    }


def ph_pairs_get_view(pairs):
    v = ph_pairs_view()
    _check(lib().ph_pairs_get_view(pairs.ptr, ctypes.byref(v)))
    return {
        "n_pairs": v.n_pairs, "n_groups": v.n_groups,
        "group_off": _dev(v.group_off, (v.n_groups + 1,), "<i8"),
        "entries": _dev(v.entries, (v.n_pairs, 4), "<f4"),
        "counts": _dev(v.counts, (v.n_pairs,), "|u1"),
        "group_order": _dev(v.group_order, (v.n_groups,), "<i4") if v.group_order else None,
    }
