"""Helpers shared by the GPU tests: a device session (params, context, keys)
through the C ABI, numpy <-> device copies, and oracle counterparts of the
synthetic workloads."""
from __future__ import annotations

import numpy as np
import torch

import paper_2509_01253_gb300 as sf
from paper_2509_01253_gb300 import workloads as wl


def to_dev(arr: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(arr)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).to("cuda")


def from_dev(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def dev_zeros(*shape) -> torch.Tensor:
    return torch.zeros(shape, dtype=torch.int64, device="cuda")


class Session:
    """Params + context + secret key (+ rotation keys) on cuda:0."""

    def __init__(self, log_n, L, bits, K, special_bits=None, sk_seed=1, rk_seed=2, rot=True, rot_d=None):
        special_bits = bits if special_bits is None else special_bits
        self.params = sf.sf_params_create(log_n, L, bits, K, special_bits, 3.2)
        self.info = sf.sf_params_get_info(self.params)
        self.n, self.L, self.K = self.info["n"], L, K
        self.ctx = sf.sf_ctx_create(self.params, 0)
        self.sk = sf.sf_keygen(self.ctx, sk_seed)
        self.rk = sf.sf_gen_rotation_keys(self.ctx, self.sk, rot_d, rk_seed) if rot else None
        self.sk_seed, self.rk_seed = sk_seed, rk_seed

    @classmethod
    def from_set(cls, ps: wl.ParamSet, **kw):
        return cls(ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits, **kw)

    def encrypt(self, msg, seed, n_cts) -> torch.Tensor:
        d = dev_zeros(n_cts, 2, self.L, self.n)
        sf.sf_encrypt(self.ctx, self.sk, msg, seed, d, n_cts)
        return d

    def decrypt(self, d, n_cts) -> np.ndarray:
        out = np.zeros((n_cts, self.L, self.n), dtype=np.uint64)
        return sf.sf_decrypt(self.ctx, self.sk, d, n_cts, out)

    def close(self):
        if self.rk:
            sf.sf_rotkeys_destroy(self.rk)
        sf.sf_secret_key_destroy(self.sk)
        sf.sf_ctx_destroy(self.ctx)
        sf.sf_params_destroy(self.params)


def oracle_params(O, log_n, L, bits, K, special_bits=None):
    return O.make_params(log_n, L, bits, K, bits if special_bits is None else special_bits)


def oracle_layer(O, case: wl.LayerCase, weight_scale: float, out_scale: float):
    terms = [O.ConvTerm(t.in_offset, t.H, t.W, t.C_in, t.C_out, t.kh, t.kw, t.stride, t.pad) for t in case.terms]
    return O.make_layer(terms, case.weights, case.bias, weight_scale, out_scale)


def gpu_layer(sess: Session, case: wl.LayerCase, weight_scale: float, out_scale: float):
    W = np.concatenate([w.ravel() for w in case.weights])
    return sf.sf_encode_weights(sess.ctx, case.terms, W, case.bias, weight_scale, out_scale)


def stream_input(case: wl.LayerCase) -> np.ndarray:
    """The client's flattened input in stream order: position k holds x[sigma_prev(k)]."""
    return case.x if case.sigma_prev is None else case.x[case.sigma_prev.astype(np.int64)]
