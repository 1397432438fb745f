"""Thin Python binding of the C ABI in include/safhire.h.

Every function has the name of the C entry point it calls and only marshals
arguments: device buffers are passed as raw pointers (ints) or objects with a
``data_ptr()`` (torch tensors), host arrays as numpy arrays, streams as
``torch.cuda.Stream`` / raw handles / None.  A non-zero status raises
:class:`SafhireError` with the library's message.  All computation happens in
the CUDA library ``_safhire.so``; there is no CPU fallback: if the library
cannot be built or loaded, or no GPU is present, the calls fail.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SF_OK, SF_EINVAL, SF_ENOMEM, SF_ECUDA, SF_ERANGE, SF_ENOTSUP = 0, 1, 2, 3, 6, 8
SF_MAX_MODULI = 12


class SafhireError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[status {status}] {message}")
        self.status = status
        self.message = message


class sf_params_info(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_int32), ("n", ctypes.c_int32), ("n_data", ctypes.c_int32),
                ("n_special", ctypes.c_int32), ("dnum", ctypes.c_int32), ("sigma", ctypes.c_double),
                ("moduli", ctypes.c_uint64 * SF_MAX_MODULI)]


class sf_conv_term(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in ("in_offset", "H", "W", "C_in", "C_out", "kh", "kw", "stride", "pad")]


class sf_layer_info(ctypes.Structure):
    _fields_ = [("E_in", ctypes.c_int32), ("E_out", ctypes.c_int32), ("k_in", ctypes.c_int32),
                ("group_size", ctypes.c_int32), ("n_groups", ctypes.c_int32), ("ks_count", ctypes.c_int64)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_u32 = ctypes.c_uint32
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_dbl = ctypes.c_double
_pp = ctypes.POINTER(ctypes.c_void_p)

_SIGS = {
    "sf_last_error": (_i32, [ctypes.c_char_p, ctypes.c_size_t]),
    "sf_version": (ctypes.c_char_p, []),
    "sf_params_create": (_i32, [_i32, _i32, _i32, _i32, _i32, _dbl, _pp]),
    "sf_params_destroy": (None, [_vp]),
    "sf_params_get_info": (_i32, [_vp, ctypes.POINTER(sf_params_info)]),
    "sf_ctx_create": (_i32, [_vp, _i32, _pp]),
    "sf_ctx_destroy": (None, [_vp]),
    "sf_ctx_set_option": (_i32, [_vp, ctypes.c_char_p, _i64]),
    "sf_ctx_get_option": (_i32, [_vp, ctypes.c_char_p, ctypes.POINTER(_i64)]),
    "sf_sync": (_i32, [_vp, _vp]),
    "sf_kernel_stats": (_i32, [_vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(_i64),
                               ctypes.POINTER(_dbl), _i32, ctypes.POINTER(_i32)]),
    "sf_kernel_stats_reset": (_i32, [_vp]),
    "sf_keygen": (_i32, [_vp, _u64, _pp]),
    "sf_secret_key_destroy": (None, [_vp]),
    "sf_secret_key_export": (_i32, [_vp, _vp]),
    "sf_gen_rotation_keys": (_i32, [_vp, _vp, _vp, _i32, _u64, _pp]),
    "sf_rotkeys_destroy": (None, [_vp]),
    "sf_rotkeys_export": (_i32, [_vp, _vp, _i32, _vp]),
    "sf_encode_input": (_i32, [_vp, _i64, _dbl, _vp]),
    "sf_client_power": (_i32, [_vp, _vp, _i32, _i32, _vp]),
    "sf_encrypt": (_i32, [_vp, _vp, _vp, _i64, _u64, _vp, _i32, _vp]),
    "sf_decrypt": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp]),
    "sf_decode": (_i32, [_vp, _vp, _i32, _i32, _i32, _dbl, _vp]),
    "sf_encode_weights": (_i32, [_vp, ctypes.POINTER(sf_conv_term), _i32, _vp, _vp, _dbl, _dbl, _pp]),
    "sf_layer_destroy": (None, [_vp]),
    "sf_layer_get_info": (_i32, [_vp, _vp, ctypes.POINTER(sf_layer_info)]),
    "sf_eval_linear_layer": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _i32, ctypes.POINTER(_i32), _vp]),
    "sf_eval_linear_layer_gamma": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _i32, _vp, _vp, _vp, _i32,
                                          ctypes.POINTER(_i32), _vp]),
    "sf_eval_linear_layer_host": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _i32, ctypes.POINTER(_i32), _vp]),
    "sf_linear_outputs": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _i32, _vp, _vp]),
    "sf_eval_layers": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sf_eval_layers_gamma": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sf_autotune_layers": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32, ctypes.POINTER(_i32),
                                  ctypes.POINTER(_dbl), _vp]),
    "sf_rotate": (_i32, [_vp, _vp, _i32, _vp, _vp, _i32, _vp]),
    "sf_rotate_noalloc": (_i32, [_vp, _vp, _i32, _vp, _vp, _i32, _vp]),
    "sf_pack": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp, _vp]),
    "sf_pack_gamma": (_i32, [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "sf_extract": (_i32, [_vp, _vp, _i32, _i32, _vp, _vp, _vp]),
    "sf_permutation": (_i32, [_u64, _u32, _u32, _vp]),
    "sf_shuffle_cts": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp]),
    "sf_poly_mul": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp]),
    "sf_ntt_batch": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp]),
    "sf_modmul_probe": (_i32, [_vp, _i32, ctypes.POINTER(_dbl)]),
    "sf_pp_ring_create": (_i32, [_i32, _i32, _i32, _i32, _i32, _pp]),
    "sf_pp_ring_destroy": (None, [_vp]),
    "sf_pp_ring_info": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), _vp]),
    "sf_pp_ntt": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp]),
    "sf_pp_mul": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp]),
    "sf_pp_automorphism": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp]),
    "sf_pp_trace": (_i32, [_vp, _vp, _vp, _i32, _i32, ctypes.POINTER(_i32), _vp]),
    "sf_pp_encrypt": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp]),
    "sf_pp_decrypt": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp]),
    "sf_pp_ksk": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, _vp]),
    "sf_pp_keyswitch": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp, _vp, _vp]),
    "sf_pp_hom_trace": (_i32, [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, ctypes.POINTER(_i32), _vp]),
    "sf_tq_ring_create": (_i32, [_i32, _i32, _i32, _i32, _i32, _pp]),
    "sf_tq_ring_destroy": (None, [_vp]),
    "sf_tq_ring_info": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), _vp, ctypes.POINTER(_i64)]),
    "sf_tq_decompose": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "sf_tq_encrypt": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp]),
    "sf_tq_decrypt": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp]),
    "sf_tq_ksk": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, _vp]),
    "sf_tq_key_prepare": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "sf_tq_keyswitch": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp, _vp]),
    "sf_tq_hom_trace": (_i32, [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp, ctypes.POINTER(_i32), _vp]),
}

_lib = None


def library_path() -> str:
    return _build.OUT


def lib() -> ctypes.CDLL:
    """Loads _safhire.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st: int):
    if st != SF_OK:
        buf = ctypes.create_string_buffer(512)
        lib().sf_last_error(buf, 512)
        raise SafhireError(st, buf.value.decode(errors="replace"))


def _ptr(x):
    """Device or host buffer -> integer address (None stays None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a buffer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    raise TypeError(f"cannot pass {type(s)} as a stream")


def _out_handle(fn, *args):
    h = ctypes.c_void_p()
    _check(fn(*args, ctypes.byref(h)))
    return h.value


# ------------------------------------------------------------------ params --

def sf_version() -> str:
    return lib().sf_version().decode()


def sf_params_create(log_n, n_data, data_bits, n_special, special_bits, sigma=3.2):
    return _out_handle(lib().sf_params_create, log_n, n_data, data_bits, n_special, special_bits, sigma)


def sf_params_destroy(p):
    lib().sf_params_destroy(p)


def sf_params_get_info(p) -> dict:
    info = sf_params_info()
    _check(lib().sf_params_get_info(p, ctypes.byref(info)))
    nm = info.n_data + info.n_special
    return {"log_n": info.log_n, "n": info.n, "n_data": info.n_data, "n_special": info.n_special,
            "dnum": info.dnum, "sigma": info.sigma, "moduli": [int(info.moduli[i]) for i in range(nm)]}


# ----------------------------------------------------------------- context --

def sf_ctx_create(params, device=0):
    return _out_handle(lib().sf_ctx_create, params, device)


def sf_ctx_destroy(ctx):
    lib().sf_ctx_destroy(ctx)


def sf_ctx_set_option(ctx, name: str, value: int):
    _check(lib().sf_ctx_set_option(ctx, name.encode(), int(value)))


def sf_ctx_get_option(ctx, name: str) -> int:
    out = _i64()
    _check(lib().sf_ctx_get_option(ctx, name.encode(), ctypes.byref(out)))
    return out.value


def sf_sync(ctx, stream=None):
    _check(lib().sf_sync(ctx, _stream(stream)))


def sf_kernel_stats(ctx) -> list:
    cap = 64
    names = (ctypes.c_char_p * cap)()
    launches = (ctypes.c_int64 * cap)()
    ms = (ctypes.c_double * cap)()
    cnt = ctypes.c_int32()
    _check(lib().sf_kernel_stats(ctx, names, launches, ms, cap, ctypes.byref(cnt)))
    return [(names[i].decode(), int(launches[i]), float(ms[i])) for i in range(min(cnt.value, cap))]


def sf_kernel_stats_reset(ctx):
    _check(lib().sf_kernel_stats_reset(ctx))


# -------------------------------------------------------------------- keys --

def sf_keygen(ctx, seed: int):
    return _out_handle(lib().sf_keygen, ctx, seed)


def sf_secret_key_destroy(sk):
    lib().sf_secret_key_destroy(sk)


def sf_secret_key_export(sk, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.int64)
    _check(lib().sf_secret_key_export(sk, _ptr(out)))
    return out


def sf_gen_rotation_keys(ctx, sk, d=None, seed=0):
    if d is None:
        return _out_handle(lib().sf_gen_rotation_keys, ctx, sk, None, 0, seed)
    arr = np.ascontiguousarray(d, dtype=np.int32)
    return _out_handle(lib().sf_gen_rotation_keys, ctx, sk, _ptr(arr), arr.size, seed)


def sf_rotkeys_destroy(rk):
    lib().sf_rotkeys_destroy(rk)


def sf_rotkeys_export(ctx, rk, d: int, out: np.ndarray) -> np.ndarray:
    _check(lib().sf_rotkeys_export(ctx, rk, d, _ptr(out)))
    return out


# ------------------------------------------------------ encrypt / decrypt --

def sf_encode_input(x, scale: float) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    out = np.zeros(x.size, dtype=np.int64)
    _check(lib().sf_encode_input(_ptr(x), x.size, scale, _ptr(out)))
    return out


def sf_client_power(params, msg, n_cts: int, d: int = 3) -> np.ndarray:
    """m(X^d) of each of n_cts chunks of N integer coefficients (Sec. 4.3)."""
    n = sf_params_get_info(params)["n"]
    m = np.zeros(n_cts * n, dtype=np.int64)
    v = np.ascontiguousarray(msg, dtype=np.int64).ravel()
    m[:v.size] = v
    out = np.zeros_like(m)
    _check(lib().sf_client_power(params, _ptr(m), n_cts, d, _ptr(out)))
    return out


def sf_encrypt(ctx, sk, msg, seed: int, d_cts, n_cts: int, stream=None):
    msg = np.ascontiguousarray(msg, dtype=np.int64).ravel()
    _check(lib().sf_encrypt(ctx, sk, _ptr(msg) if msg.size else None, msg.size, seed, _ptr(d_cts), n_cts,
                            _stream(stream)))


def sf_decrypt(ctx, sk, d_cts, n_cts: int, out: np.ndarray, stream=None) -> np.ndarray:
    if out.dtype != np.uint64:
        raise TypeError("residues are uint64")
    _check(lib().sf_decrypt(ctx, sk, _ptr(d_cts), n_cts, _ptr(out), _stream(stream)))
    return out


def sf_decode(params, residues: np.ndarray, n_cts: int, stride: int, count: int, scale: float) -> np.ndarray:
    residues = np.ascontiguousarray(residues, dtype=np.uint64)
    out = np.zeros(count, dtype=np.float64)
    _check(lib().sf_decode(params, _ptr(residues), n_cts, stride, count, scale, _ptr(out)))
    return out


# ------------------------------------------------------------------ layers --

def _terms(terms):
    arr = (sf_conv_term * len(terms))()
    for i, t in enumerate(terms):
        if isinstance(t, dict):
            vals = [t.get(f, 0 if f in ("in_offset", "pad") else 1) for f, _ in sf_conv_term._fields_]
        else:
            vals = [getattr(t, f, 0 if f in ("in_offset", "pad") else 1) for f, _ in sf_conv_term._fields_]
        for (f, _), v in zip(sf_conv_term._fields_, vals):
            setattr(arr[i], f, int(v))
    return arr


def sf_encode_weights(ctx, terms, W, bias, weight_scale: float, bias_scale: float = 0.0):
    arr = _terms(terms)
    w = np.ascontiguousarray(W, dtype=np.float64).ravel()
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float64).ravel()
    return _out_handle(lib().sf_encode_weights, ctx, arr, len(terms), _ptr(w), _ptr(b), weight_scale, bias_scale)


def sf_layer_destroy(layer):
    lib().sf_layer_destroy(layer)


def sf_layer_get_info(ctx, layer) -> dict:
    info = sf_layer_info()
    _check(lib().sf_layer_get_info(ctx, layer, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in sf_layer_info._fields_}


def _perm(p):
    return None if p is None else np.ascontiguousarray(p, dtype=np.uint32)


def sf_eval_linear_layer(ctx, layer, rk, d_in, k_in: int, sigma_prev, sigma_out, d_out, out_capacity: int,
                         stream=None) -> int:
    sp, so = _perm(sigma_prev), _perm(sigma_out)
    n_out = ctypes.c_int32()
    _check(lib().sf_eval_linear_layer(ctx, layer, rk, _ptr(d_in), k_in, _ptr(sp), _ptr(so), _ptr(d_out),
                                      out_capacity, ctypes.byref(n_out), _stream(stream)))
    return n_out.value


def sf_eval_linear_layer_gamma(ctx, layer, rk, gamma: int, d_in, d_powers, k_in: int, sigma_prev, sigma_out, d_out,
                               out_capacity: int, stream=None) -> int:
    sp, so = _perm(sigma_prev), _perm(sigma_out)
    n_out = ctypes.c_int32()
    _check(lib().sf_eval_linear_layer_gamma(ctx, layer, rk, gamma, _ptr(d_in), _ptr(d_powers), k_in, _ptr(sp),
                                            _ptr(so), _ptr(d_out), out_capacity, ctypes.byref(n_out), _stream(stream)))
    return n_out.value


def sf_eval_linear_layer_host(ctx, layer, rk, h_in: np.ndarray, k_in: int, sigma_prev, sigma_out, h_out: np.ndarray,
                              out_capacity: int, stream=None) -> int:
    sp, so = _perm(sigma_prev), _perm(sigma_out)
    n_out = ctypes.c_int32()
    _check(lib().sf_eval_linear_layer_host(ctx, layer, rk, _ptr(h_in), k_in, _ptr(sp), _ptr(so), _ptr(h_out),
                                           out_capacity, ctypes.byref(n_out), _stream(stream)))
    return n_out.value


def _round_arrays(layers, rks, d_ins, k_ins, sigma_prevs, sigma_outs, d_outs, out_capacities):
    n = len(layers)
    VP = ctypes.c_void_p * n
    keep = []
    def perms(ps):
        if ps is None:
            return None
        arr = VP()
        for i, p in enumerate(ps):
            pp = _perm(p)
            keep.append(pp)
            arr[i] = _ptr(pp) if pp is not None else None
        return arr
    a = (VP(*layers), VP(*rks), VP(*[_ptr(x) for x in d_ins]), (ctypes.c_int32 * n)(*k_ins), perms(sigma_prevs),
         perms(sigma_outs), VP(*[_ptr(x) for x in d_outs]), (ctypes.c_int32 * n)(*out_capacities))
    return a, keep


def sf_eval_layers(ctx, layers, rks, d_ins, k_ins, sigma_prevs, sigma_outs, d_outs, out_capacities, stream=None):
    """Several layer rounds in one captured launch sequence; returns n_outs."""
    a, keep = _round_arrays(layers, rks, d_ins, k_ins, sigma_prevs, sigma_outs, d_outs, out_capacities)
    n_outs = (ctypes.c_int32 * len(layers))()
    _check(lib().sf_eval_layers(ctx, len(layers), *a, n_outs, _stream(stream)))
    return list(n_outs)


def sf_eval_layers_gamma(ctx, layers, rks, d_ins, d_powers, k_ins, sigma_prevs, sigma_outs, d_outs, out_capacities,
                         stream=None):
    """sf_eval_layers where round x runs at gamma = 2 when d_powers[x] is a
    buffer of the client's powers (None: gamma = 0); returns n_outs."""
    a, keep = _round_arrays(layers, rks, d_ins, k_ins, sigma_prevs, sigma_outs, d_outs, out_capacities)
    n = len(layers)
    pw = None if d_powers is None else (ctypes.c_void_p * n)(*[_ptr(x) for x in d_powers])
    n_outs = (ctypes.c_int32 * n)()
    _check(lib().sf_eval_layers_gamma(ctx, n, a[0], a[1], a[2], pw, *a[3:], n_outs, _stream(stream)))
    return list(n_outs)


def sf_autotune_layers(ctx, layers, rks, d_ins, k_ins, sigma_prevs, sigma_outs, d_outs, out_capacities, repeats=2,
                       stream=None):
    """Chooses the key-switch launch batch by timing; returns (ks_batch, ms)."""
    a, keep = _round_arrays(layers, rks, d_ins, k_ins, sigma_prevs, sigma_outs, d_outs, out_capacities)
    best = ctypes.c_int32()
    ms = ctypes.c_double()
    _check(lib().sf_autotune_layers(ctx, len(layers), *a, repeats, ctypes.byref(best), ctypes.byref(ms),
                                    _stream(stream)))
    return best.value, ms.value


def sf_linear_outputs(ctx, layer, d_in, k_in: int, sigma_prev, outputs, d_out, stream=None):
    sp = _perm(sigma_prev)
    outs = np.ascontiguousarray(outputs, dtype=np.int32)
    _check(lib().sf_linear_outputs(ctx, layer, _ptr(d_in), k_in, _ptr(sp), _ptr(outs), outs.size, _ptr(d_out),
                                   _stream(stream)))


# --------------------------------------------------------- building blocks --

def sf_rotate(ctx, rk, d: int, d_ct, d_out, count: int, stream=None):
    _check(lib().sf_rotate(ctx, rk, d, _ptr(d_ct), _ptr(d_out), count, _stream(stream)))


def sf_rotate_noalloc(ctx, rk, d: int, d_ct, d_out, count: int, stream=None):
    """sf_rotate without any device allocation (fixed 32 MiB scratch compiled
    into the library; see include/safhire.h for the limits)."""
    _check(lib().sf_rotate_noalloc(ctx, rk, d, _ptr(d_ct), _ptr(d_out), count, _stream(stream)))


def sf_pack(ctx, rk, d_leaves, n_leaves: int, n: int, d_out, stream=None):
    _check(lib().sf_pack(ctx, rk, _ptr(d_leaves), n_leaves, n, _ptr(d_out), _stream(stream)))


def sf_pack_gamma(ctx, rk, d_leaves, n_leaves: int, n: int, gamma: int, d_out, stream=None):
    _check(lib().sf_pack_gamma(ctx, rk, _ptr(d_leaves), n_leaves, n, gamma, _ptr(d_out), _stream(stream)))


def sf_extract(ctx, d_ct, i: int, gamma: int, d_powers, d_out, stream=None):
    _check(lib().sf_extract(ctx, _ptr(d_ct), i, gamma, _ptr(d_powers), _ptr(d_out), _stream(stream)))


def sf_permutation(session_seed: int, rnd: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint32)
    _check(lib().sf_permutation(session_seed, rnd, n, _ptr(out) if n else None))
    return out


def sf_shuffle_cts(ctx, perm, d_in, d_out, count: int, stream=None):
    p = _perm(perm)
    _check(lib().sf_shuffle_cts(ctx, _ptr(p), _ptr(d_in), _ptr(d_out), count, _stream(stream)))


def sf_poly_mul(ctx, d_a, d_b, d_out, n_polys: int, stream=None):
    _check(lib().sf_poly_mul(ctx, _ptr(d_a), _ptr(d_b), _ptr(d_out), n_polys, _stream(stream)))


def sf_ntt_batch(ctx, d_in, d_out, count: int, inverse: bool, stream=None):
    _check(lib().sf_ntt_batch(ctx, _ptr(d_in), _ptr(d_out), count, 1 if inverse else 0, _stream(stream)))


def sf_modmul_probe(ctx, kind: int) -> float:
    """Measured modular-multiplication rate (10^9/s) of kind 0 (forward
    butterfly), 1 (inverse butterfly) or 2 (multiply-accumulate)."""
    out = _dbl()
    _check(lib().sf_modmul_probe(ctx, kind, ctypes.byref(out)))
    return out.value


EXPORTED = sorted(_SIGS)


# ---------------------------------------------------- prime-power rings --

def sf_pp_ring_create(t: int, alpha: int, L: int, bits: int, device: int = 0):
    return _out_handle(lib().sf_pp_ring_create, t, alpha, L, bits, device)


def sf_pp_ring_destroy(r):
    lib().sf_pp_ring_destroy(r)


def sf_pp_ring_info(r, L: int) -> dict:
    n, m = _i32(), _i32()
    mods = np.zeros(L, dtype=np.uint64)
    _check(lib().sf_pp_ring_info(r, ctypes.byref(n), ctypes.byref(m), mods.ctypes.data))
    return {"N": n.value, "M": m.value, "moduli": [int(q) for q in mods]}


def sf_pp_ntt(r, d_in, d_out, count: int, inverse: bool, stream=None):
    _check(lib().sf_pp_ntt(r, _ptr(d_in), _ptr(d_out), count, 1 if inverse else 0, _stream(stream)))


def sf_pp_mul(r, d_a, d_b, d_out, count: int, stream=None):
    _check(lib().sf_pp_mul(r, _ptr(d_a), _ptr(d_b), _ptr(d_out), count, _stream(stream)))


def sf_pp_automorphism(r, d_in, d_out, count: int, d: int, stream=None):
    _check(lib().sf_pp_automorphism(r, _ptr(d_in), _ptr(d_out), count, d, _stream(stream)))


def sf_pp_trace(r, d_in, d_out, count: int, gamma: int, stream=None) -> int:
    """Returns the number of automorphisms applied."""
    n = _i32()
    _check(lib().sf_pp_trace(r, _ptr(d_in), _ptr(d_out), count, gamma, ctypes.byref(n), _stream(stream)))
    return n.value


def sf_pp_encrypt(r, d_s, d_a, d_m, d_e, d_ct, count: int, stream=None):
    _check(lib().sf_pp_encrypt(r, _ptr(d_s), _ptr(d_a), _ptr(d_m), _ptr(d_e), _ptr(d_ct), count, _stream(stream)))


def sf_pp_decrypt(r, d_s, d_ct, d_out, count: int, stream=None):
    _check(lib().sf_pp_decrypt(r, _ptr(d_s), _ptr(d_ct), _ptr(d_out), count, _stream(stream)))


def sf_pp_ksk(r, d_s, h: int, d_ka, d_e, d_kb, stream=None):
    _check(lib().sf_pp_ksk(r, _ptr(d_s), h, _ptr(d_ka), _ptr(d_e), _ptr(d_kb), _stream(stream)))


def sf_pp_keyswitch(r, d_ct, d_out, count: int, h: int, d_ka, d_kb, stream=None):
    _check(lib().sf_pp_keyswitch(r, _ptr(d_ct), _ptr(d_out), count, h, _ptr(d_ka), _ptr(d_kb), _stream(stream)))


def sf_pp_hom_trace(r, d_ct, d_out, count: int, gamma: int, keys: dict, stream=None) -> int:
    """keys: {h: (d_ka, d_kb)}.  Returns the number of key switches run."""
    hs = sorted(keys)
    H = (_i32 * max(1, len(hs)))(*hs)
    KA = (_vp * max(1, len(hs)))(*[_ptr(keys[h][0]) for h in hs])
    KB = (_vp * max(1, len(hs)))(*[_ptr(keys[h][1]) for h in hs])
    n = _i32()
    _check(lib().sf_pp_hom_trace(r, _ptr(d_ct), _ptr(d_out), count, gamma, len(hs), ctypes.cast(H, _vp),
                                 ctypes.cast(KA, _vp), ctypes.cast(KB, _vp), ctypes.byref(n), _stream(stream)))
    return n.value


# ------------------------------------- torus scheme (q = 2^53, gadget D, l) --

def sf_tq_ring_create(t: int, alpha: int, D: int, l: int, device: int = 0):
    return _out_handle(lib().sf_tq_ring_create, t, alpha, D, l, device)


def sf_tq_ring_destroy(r):
    lib().sf_tq_ring_destroy(r)


def sf_tq_ring_info(r) -> dict:
    n, m, kw = _i32(), _i32(), _i64()
    primes = np.zeros(2, dtype=np.uint64)
    _check(lib().sf_tq_ring_info(r, ctypes.byref(n), ctypes.byref(m), primes.ctypes.data, ctypes.byref(kw)))
    return {"N": n.value, "M": m.value, "primes": [int(p) for p in primes], "key_words": kw.value}


def sf_tq_decompose(r, d_in, d_digits, count: int, stream=None):
    _check(lib().sf_tq_decompose(r, _ptr(d_in), _ptr(d_digits), count, _stream(stream)))


def sf_tq_encrypt(r, d_s, d_a, d_m, d_e, d_ct, count: int, stream=None):
    _check(lib().sf_tq_encrypt(r, _ptr(d_s), _ptr(d_a), _ptr(d_m), _ptr(d_e), _ptr(d_ct), count, _stream(stream)))


def sf_tq_decrypt(r, d_s, d_ct, d_phase, count: int, stream=None):
    _check(lib().sf_tq_decrypt(r, _ptr(d_s), _ptr(d_ct), _ptr(d_phase), count, _stream(stream)))


def sf_tq_ksk(r, d_s, h: int, d_ka, d_e, d_kb, stream=None):
    _check(lib().sf_tq_ksk(r, _ptr(d_s), h, _ptr(d_ka), _ptr(d_e), _ptr(d_kb), _stream(stream)))


def sf_tq_key_prepare(r, d_ka, d_kb, d_key, stream=None):
    _check(lib().sf_tq_key_prepare(r, _ptr(d_ka), _ptr(d_kb), _ptr(d_key), _stream(stream)))


def sf_tq_keyswitch(r, d_ct, d_out, count: int, h: int, d_key, stream=None):
    _check(lib().sf_tq_keyswitch(r, _ptr(d_ct), _ptr(d_out), count, h, _ptr(d_key), _stream(stream)))


def sf_tq_hom_trace(r, d_ct, d_out, count: int, gamma: int, keys: dict, stream=None) -> int:
    """keys: {h: d_key (prepared)}.  Returns the number of key switches run."""
    hs = sorted(keys)
    H = (_i32 * max(1, len(hs)))(*hs)
    K = (_vp * max(1, len(hs)))(*[_ptr(keys[h]) for h in hs])
    n = _i32()
    _check(lib().sf_tq_hom_trace(r, _ptr(d_ct), _ptr(d_out), count, gamma, len(hs), ctypes.cast(H, _vp),
                                 ctypes.cast(K, _vp), ctypes.byref(n), _stream(stream)))
    return n.value
