"""Plain CPU oracle for the Safhire server-side linear-layer round.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package.  The product path
(``paper_2509_01253_gb300``) never imports it, and the two share no code: the
arithmetic here lives in ``oracle.c`` (schoolbook negacyclic products, direct
automorphisms, textbook hybrid key switching) and in the short recursions
below, which follow the paper's algorithms step by step:

* Sec. 2.1   RLWE over Z_Q[X]/(X^N+1) (the cyclotomic Phi_M at t = 2, M = 2N)
* Sec. 2.2   automorphism X -> X^d followed by key switching
* Sec. 2.3   trace, evaluated as a tower of automorphism-and-add steps
* Sec. 2.4   packing: PackLWEs tree, then the field trace that zeroes all
             non-packed coefficients
* Sec. 4.4   server round: extraction (gamma = 0, and gamma = 2 from the
             client's power m(X^3), Lemma 1 at t = 2), unshuffle, linear layer,
             shuffle, fast packing

Parity status of every function: pinned by tests/test_oracle_pins.py (see the
docstring of each test for the independent fact it checks).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_dblp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.or_is_prime.restype = ctypes.c_int
        L.or_is_prime.argtypes = [ctypes.c_uint64]
        L.or_find_primes.restype = ctypes.c_int
        L.or_find_primes.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _u64p]
        L.or_primitive_root_2n.restype = ctypes.c_uint64
        L.or_primitive_root_2n.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.or_mulmod.restype = ctypes.c_uint64
        L.or_mulmod.argtypes = [ctypes.c_uint64] * 3
        L.or_invmod.restype = ctypes.c_uint64
        L.or_invmod.argtypes = [ctypes.c_uint64] * 2
        L.or_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_int64, _u64p]
        L.or_sample_secret.argtypes = [ctypes.c_uint64, ctypes.c_int, _i64p]
        L.or_sample_encrypt.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _u64p,
                                        ctypes.c_int, ctypes.c_double, _u64p, _i64p]
        L.or_sample_rotkey.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, _u64p, ctypes.c_double, _u64p, _i64p]
        L.or_permutation.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _u32p]
        L.or_quantize.argtypes = [_dblp, ctypes.c_int64, ctypes.c_double, _i64p]
        L.or_polymul.argtypes = [_u64p, _u64p, _u64p, ctypes.c_int, ctypes.c_uint64]
        L.or_automorphism.argtypes = [_u64p, _u64p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64]
        L.or_monomial_mul.argtypes = [_u64p, _u64p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64]
        L.or_encrypt.argtypes = [ctypes.c_int, ctypes.c_int, _u64p, _i64p, _i64p, _u64p, _i64p, _u64p]
        L.or_decrypt.argtypes = [ctypes.c_int, ctypes.c_int, _u64p, _i64p, _u64p, _u64p, _u64p]
        L.or_modup.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _u64p, ctypes.c_int, _u64p, _u64p]
        L.or_moddown.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _u64p, _u64p, _u64p]
        L.or_rotkey.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _u64p, ctypes.c_int64,
                                _i64p, _u64p, _i64p, _u64p]
        L.or_keyswitch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _u64p, _u64p, _u64p,
                                   _u64p, _u64p]
        L.or_rotate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _u64p, _u64p, ctypes.c_int64,
                                _u64p, _u64p]
        L.or_linear_output.argtypes = [ctypes.c_int, ctypes.c_int, _u64p, ctypes.c_int, _u64p,
                                       ctypes.c_int, _i64p, _i64p, _u64p]
    return _lib


def _p(a: np.ndarray, ptype):
    return a.ctypes.data_as(ptype)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int64)


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------

@dataclass
class Params:
    """RNS parameters: data primes q_0..q_{L-1} (Q), special primes p_0..p_{K-1} (P).

    Digit j of the hybrid gadget holds data limbs [jK, min((j+1)K, L))."""
    log_n: int
    n: int
    L: int
    K: int
    q: list
    p: list
    sigma: float = 3.2

    @property
    def mods(self) -> list:
        return list(self.q) + list(self.p)

    @property
    def dnum(self) -> int:
        return (self.L + self.K - 1) // self.K

    @property
    def Q(self) -> int:
        return math.prod(self.q)

    @property
    def P(self) -> int:
        return math.prod(self.p)

    def digit(self, j: int) -> range:
        return range(j * self.K, min((j + 1) * self.K, self.L))


def find_primes(two_n: int, bits: int, count: int) -> list:
    out = np.zeros(count, dtype=np.uint64)
    got = lib().or_find_primes(two_n, bits, count, _p(out, _u64p))
    assert got == count
    return [int(x) for x in out]


def make_params(log_n: int, L: int, data_bits: int, K: int, special_bits: int,
                sigma: float = 3.2) -> Params:
    """Primes q = 1 mod 2N, descending from 2^bits.  When data and special
    primes have the same size the first K found are the special primes and the
    next L the data primes; otherwise each set is the top of its own size."""
    n = 1 << log_n
    if data_bits == special_bits:
        pr = find_primes(2 * n, data_bits, K + L)
        p, q = pr[:K], pr[K:]
    else:
        p = find_primes(2 * n, special_bits, K)
        cand = find_primes(2 * n, data_bits, L + K)
        q = [c for c in cand if c not in p][:L]
    return Params(log_n=log_n, n=n, L=L, K=K, q=q, p=p, sigma=sigma)


# ---------------------------------------------------------------------------
# samplers (SplitMix64 / Lemire / Box-Muller; each side implements its own)
# ---------------------------------------------------------------------------

def splitmix64(seed: int, count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.uint64)
    lib().or_splitmix64(seed, count, _p(out, _u64p))
    return out


def keygen(prm: Params, seed: int) -> np.ndarray:
    s = np.zeros(prm.n, dtype=np.int64)
    lib().or_sample_secret(seed, prm.n, _p(s, _i64p))
    return s


def permutation(session_seed: int, rnd: int, n: int) -> np.ndarray:
    perm = np.zeros(n, dtype=np.uint32)
    lib().or_permutation(session_seed, rnd, n, _p(perm, _u32p))
    return perm


def quantize(x, scale: float) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    out = np.zeros(x.size, dtype=np.int64)
    lib().or_quantize(_p(x, _dblp), x.size, scale, _p(out, _i64p))
    return out


def sample_encrypt(prm: Params, seed: int, n_cts: int):
    q = _u64(prm.q)
    a = np.zeros((n_cts, prm.L, prm.n), dtype=np.uint64)
    e = np.zeros((n_cts, prm.n), dtype=np.int64)
    lib().or_sample_encrypt(seed, prm.n, prm.L, _p(q, _u64p), n_cts, prm.sigma, _p(a, _u64p), _p(e, _i64p))
    return a, e


# ---------------------------------------------------------------------------
# ring and RLWE primitives
# ---------------------------------------------------------------------------

def polymul(a, b, q: int) -> np.ndarray:
    a, b = _u64(a), _u64(b)
    c = np.zeros_like(a)
    lib().or_polymul(_p(a, _u64p), _p(b, _u64p), _p(c, _u64p), a.size, q)
    return c


def automorphism(a, d: int, q: int) -> np.ndarray:
    a = _u64(a)
    out = np.zeros_like(a)
    lib().or_automorphism(_p(a, _u64p), _p(out, _u64p), a.size, d, q)
    return out


def monomial_mul(a, s: int, q: int) -> np.ndarray:
    a = _u64(a)
    out = np.zeros_like(a)
    lib().or_monomial_mul(_p(a, _u64p), _p(out, _u64p), a.size, s, q)
    return out


def encrypt(prm: Params, s: np.ndarray, msg, seed: int, n_cts: int) -> np.ndarray:
    """Sec. 2.1: RLWE_s(m) = (a, a*s + m + e) per chunk of N message values
    (Sec. 4.3 "Flatten and chunk": chunk j holds msg[jN:(j+1)N], zero-padded)."""
    msg = _i64(msg).ravel()
    assert msg.size <= n_cts * prm.n
    m = np.zeros(n_cts * prm.n, dtype=np.int64)
    m[:msg.size] = msg
    a, e = sample_encrypt(prm, seed, n_cts)
    q = _u64(prm.q)
    s = _i64(s)
    cts = np.zeros((n_cts, 2, prm.L, prm.n), dtype=np.uint64)
    for j in range(n_cts):
        cts[j, 0] = a[j]
        b = np.zeros((prm.L, prm.n), dtype=np.uint64)
        mj = np.ascontiguousarray(m[j * prm.n:(j + 1) * prm.n])
        ej = np.ascontiguousarray(e[j])
        aj = np.ascontiguousarray(a[j])
        lib().or_encrypt(prm.n, prm.L, _p(q, _u64p), _p(s, _i64p), _p(mj, _i64p), _p(aj, _u64p),
                         _p(ej, _i64p), _p(b, _u64p))
        cts[j, 1] = b
    return cts


def decrypt(prm: Params, s: np.ndarray, cts: np.ndarray) -> np.ndarray:
    """Plaintext residues b - a*s, shape [n_cts][L][N]."""
    cts = _u64(cts).reshape(-1, 2, prm.L, prm.n)
    q = _u64(prm.q)
    s = _i64(s)
    out = np.zeros((cts.shape[0], prm.L, prm.n), dtype=np.uint64)
    for j in range(cts.shape[0]):
        a = np.ascontiguousarray(cts[j, 0])
        b = np.ascontiguousarray(cts[j, 1])
        m = np.zeros((prm.L, prm.n), dtype=np.uint64)
        lib().or_decrypt(prm.n, prm.L, _p(q, _u64p), _p(s, _i64p), _p(a, _u64p), _p(b, _u64p), _p(m, _u64p))
        out[j] = m
    return out


def crt_centered(prm: Params, residues: np.ndarray) -> list:
    """CRT of [L][...] residues into centred integers in (-Q/2, Q/2] (Python ints)."""
    Q = prm.Q
    res = np.asarray(residues).reshape(prm.L, -1)
    coefs = []
    for i, qi in enumerate(prm.q):
        qhat = Q // qi
        coefs.append(qhat * pow(qhat % qi, -1, qi))
    out = []
    for k in range(res.shape[1]):
        v = sum(int(res[i, k]) * coefs[i] for i in range(prm.L)) % Q
        if v > Q // 2:
            v -= Q
        out.append(v)
    return out


def decode(prm: Params, residues: np.ndarray, scale: float) -> np.ndarray:
    """Centred CRT value / scale, as float64 (exact division in Python ints
    first, so no precision is lost for values far above 2^53)."""
    vals = crt_centered(prm, residues)
    return np.array([float(v) / scale for v in vals], dtype=np.float64)


# ---------------------------------------------------------------------------
# key switching
# ---------------------------------------------------------------------------

def sample_rotkey(prm: Params, seed: int, d: int):
    mods = _u64(prm.mods)
    nm = prm.L + prm.K
    alpha = np.zeros((prm.dnum, nm, prm.n), dtype=np.uint64)
    e = np.zeros((prm.dnum, prm.n), dtype=np.int64)
    lib().or_sample_rotkey(seed, d, prm.n, prm.dnum, nm, _p(mods, _u64p), prm.sigma,
                           _p(alpha, _u64p), _p(e, _i64p))
    return alpha, e


def rotkey(prm: Params, s: np.ndarray, seed: int, d: int) -> np.ndarray:
    """Key for tau_d, layout [dnum][2][L+K][N] (coefficient domain)."""
    alpha, e = sample_rotkey(prm, seed, d)
    mods = _u64(prm.mods)
    key = np.zeros((prm.dnum, 2, prm.L + prm.K, prm.n), dtype=np.uint64)
    lib().or_rotkey(prm.n, prm.L, prm.K, _p(mods, _u64p), d, _p(_i64(s), _i64p),
                    _p(alpha, _u64p), _p(e, _i64p), _p(key, _u64p))
    return key


def default_rotation_indices(prm: Params) -> list:
    """d = 2^k + 1 for k = 1..log2 N: every automorphism the packing tree and
    the field trace use (Sec. 4.2: at most alpha(t-1) = log2(2N) indices)."""
    return [(1 << k) + 1 for k in range(1, prm.log_n + 1)]


def rotation_keys(prm: Params, s: np.ndarray, seed: int, indices=None) -> dict:
    idx = default_rotation_indices(prm) if indices is None else list(indices)
    return {d: rotkey(prm, s, seed, d) for d in idx}


def modup(prm: Params, j: int, x: np.ndarray) -> np.ndarray:
    x = _u64(x).reshape(prm.L, prm.n)
    mods = _u64(prm.mods)
    out = np.zeros((prm.L + prm.K, prm.n), dtype=np.uint64)
    lib().or_modup(prm.n, prm.L, prm.K, _p(mods, _u64p), j, _p(x, _u64p), _p(out, _u64p))
    return out


def moddown(prm: Params, x: np.ndarray) -> np.ndarray:
    x = _u64(x).reshape(prm.L + prm.K, prm.n)
    mods = _u64(prm.mods)
    out = np.zeros((prm.L, prm.n), dtype=np.uint64)
    lib().or_moddown(prm.n, prm.L, prm.K, _p(mods, _u64p), _p(x, _u64p), _p(out, _u64p))
    return out


def keyswitch(prm: Params, key: np.ndarray, c: np.ndarray):
    mods = _u64(prm.mods)
    c = _u64(c).reshape(prm.L, prm.n)
    A = np.zeros((prm.L, prm.n), dtype=np.uint64)
    B = np.zeros((prm.L, prm.n), dtype=np.uint64)
    lib().or_keyswitch(prm.n, prm.L, prm.K, _p(mods, _u64p), _p(_u64(key), _u64p), _p(c, _u64p),
                       _p(A, _u64p), _p(B, _u64p))
    return A, B


class Counter:
    """Counts key switches (one per rotate)."""

    def __init__(self):
        self.ks = 0


def rotate(prm: Params, keys: dict, d: int, ct: np.ndarray, counter: Counter | None = None) -> np.ndarray:
    """tau_d then key switching back to s(X) (Sec. 2.2)."""
    if d not in keys:
        raise KeyError(f"no rotation key for d={d}")
    mods = _u64(prm.mods)
    ct = _u64(ct).reshape(2, prm.L, prm.n)
    out = np.zeros_like(ct)
    lib().or_rotate(prm.n, prm.L, prm.K, _p(mods, _u64p), _p(_u64(keys[d]), _u64p), d,
                    _p(ct, _u64p), _p(out, _u64p))
    if counter is not None:
        counter.ks += 1
    return out


# ---------------------------------------------------------------------------
# ciphertext arithmetic used by the packing recursion
# ---------------------------------------------------------------------------

def _qcol(prm: Params) -> np.ndarray:
    return np.array(prm.q, dtype=np.uint64).reshape(1, prm.L, 1)


def ct_add(prm: Params, x, y) -> np.ndarray:
    q = _qcol(prm)
    return (_u64(x) + _u64(y)) % q


def ct_sub(prm: Params, x, y) -> np.ndarray:
    q = _qcol(prm)
    return (_u64(x) + (q - _u64(y))) % q


def ct_monomial(prm: Params, ct, s: int) -> np.ndarray:
    ct = _u64(ct).reshape(2, prm.L, prm.n)
    out = np.zeros_like(ct)
    for part in range(2):
        for i in range(prm.L):
            out[part, i] = monomial_mul(ct[part, i], s, prm.q[i])
    return out


def zero_ct(prm: Params) -> np.ndarray:
    return np.zeros((2, prm.L, prm.n), dtype=np.uint64)


# ---------------------------------------------------------------------------
# packing (Sec. 2.4; Sec. 4.4 "Fast Packing") at t = 2
# ---------------------------------------------------------------------------

def pack_tree(prm: Params, keys: dict, leaves: list, counter: Counter | None = None,
              gamma: int = 0) -> np.ndarray:
    """PackLWEs recursion on n = 2^k ciphertexts:
        Pack(ct_0..ct_{n-1}) = (E + X^{N/n} O) + tau_{n+1}(E - X^{N/n} O)
    with E = Pack(even-indexed), O = Pack(odd-indexed), tau followed by key
    switching.  Coefficient 0 of leaf l ends, times n, at X^{l N/n}.

    gamma = 2 (Sec. 4.4, Lemma 1 at t = 2): each leaf already encrypts
    y + tau_3(y), its image under the partial trace over K_2 / K_0 (the
    automorphisms {1, 3}).  The merge of two leaves is then
    (E + tau_3 E) + X^{N/2} (O + tau_3 O) = E' + X^{N/2} O' with no key
    switch: the level whose automorphism tau_3 the client has applied."""
    n = len(leaves)
    assert n >= 1 and (n & (n - 1)) == 0
    if n == 1:
        return _u64(leaves[0]).reshape(2, prm.L, prm.n)
    E = pack_tree(prm, keys, leaves[0::2], counter, gamma)
    O = pack_tree(prm, keys, leaves[1::2], counter, gamma)
    XO = ct_monomial(prm, O, prm.n // n)
    if gamma == 2 and n == 2:
        return ct_add(prm, E, XO)
    return ct_add(prm, ct_add(prm, E, XO), rotate(prm, keys, n + 1, ct_sub(prm, E, XO), counter))


def field_trace(prm: Params, keys: dict, ct: np.ndarray, n: int, counter: Counter | None = None,
                gamma: int = 0) -> np.ndarray:
    """The remaining trace levels after packing n values (Sec. 2.3, 2.4):
    for k = log2(n)+1 .. log2(N):  ct <- ct + tau_{2^k+1}(ct).  Zeroes every
    coefficient outside the stride-N/n lattice and multiplies the rest by N/n.
    gamma = 2 with a single value (n = 1) starts at k = 2: the client's
    partial trace supplied the tau_3 step (Tr over K_2 / K_1)."""
    k0 = int(math.log2(n))
    start = max(k0 + 1, 2) if gamma == 2 else k0 + 1
    for k in range(start, prm.log_n + 1):
        ct = ct_add(prm, ct, rotate(prm, keys, (1 << k) + 1, ct, counter))
    return ct


def pack(prm: Params, keys: dict, leaves: list, counter: Counter | None = None,
         n: int | None = None, gamma: int = 0) -> np.ndarray:
    """Fast packing of len(leaves) <= n <= N/2 ciphertexts, zero-padded to n
    (default: the next power of two): output coefficient l*N/n holds
    N * (coefficient 0 of leaf l) at gamma = 0, and N * (coefficient 0 of y_l)
    at gamma = 2 when leaf l encrypts y_l + tau_3(y_l)."""
    assert gamma in (0, 2)
    m = len(leaves)
    if n is None:
        n = 1
        while n < m:
            n *= 2
    assert m <= n and (n & (n - 1)) == 0
    assert n <= prm.n // 2, "at t = 2 a ciphertext packs at most N/2 values (beta <= alpha - 1)"
    leaves = list(leaves) + [zero_ct(prm)] * (n - m)
    return field_trace(prm, keys, pack_tree(prm, keys, leaves, counter, gamma), n, counter, gamma)


def group_size(prm: Params, e_out: int) -> int:
    """Values per packed ciphertext: min(N/2, next power of two >= E')."""
    n = 1
    while n < e_out:
        n *= 2
    return min(prm.n // 2, n)


def ks_count(prm: Params, e_out: int, gamma: int = 0) -> int:
    """Key switches for one layer round: per group (n - 1) tree merges plus
    log2(N/n) trace steps; at gamma = 2 the tau_3 level costs none (n/2 merges
    of the bottom level, or the first trace step when n = 1)."""
    n = group_size(prm, e_out)
    groups = -(-e_out // n)
    per = (n - 1) + (prm.log_n - int(math.log2(n)))
    if gamma == 2:
        per -= n // 2 if n >= 2 else 1
    return groups * per


def ks_per_coefficient_general(t: int, alpha: int, gamma: int) -> float:
    """Key switches per packed coefficient for M = t^alpha (Sec. 2.4, Table 1):
    sum_{l in omega_{t-1}} (l - 1) + sum_{1<=i<=alpha} t^-(i-1), with the
    first term dropped for gamma >= 1 and the i = 1 term dropped for gamma = 2
    (the client supplies the partial traces Tr_{K1/K0} and Tr_{K2/K1})."""
    def prime_factors(x):
        f, d = [], 2
        while d * d <= x:
            while x % d == 0:
                f.append(d)
                x //= d
            d += 1
        if x > 1:
            f.append(x)
        return f
    first = sum(l - 1 for l in prime_factors(t - 1)) if t > 2 else 0
    tail = [t ** -(i - 1) for i in range(1, alpha + 1)]
    if gamma >= 1:
        first = 0
    if gamma >= 2:
        tail = tail[1:]
    return first + sum(tail)


# ---------------------------------------------------------------------------
# linear layer (Sec. 4.4 steps 6-8)
# ---------------------------------------------------------------------------

@dataclass
class ConvTerm:
    """One linear term of a layer: a convolution over an input segment.
    Input segment: H x W x C_in, flattened row-major with channels last
    (Sec. 4.3), starting at flat index in_offset of the layer input.
    FC layers are 1x1 inputs with 1x1 kernels; a global-average-pooled FC is a
    kernel as large as the input."""
    in_offset: int
    H: int
    W: int
    C_in: int
    C_out: int
    kh: int
    kw: int
    stride: int = 1
    pad: int = 0

    @property
    def H_out(self):
        return (self.H + 2 * self.pad - self.kh) // self.stride + 1

    @property
    def W_out(self):
        return (self.W + 2 * self.pad - self.kw) // self.stride + 1


@dataclass
class Layer:
    terms: list
    weights: list            # per term, float64 [C_out][kh][kw][C_in]
    bias: np.ndarray | None = None   # float64 [C_out] or None
    E_in: int = 0
    quantized: list = field(default_factory=list)   # per term, int64 weights
    bias_q: np.ndarray | None = None

    @property
    def H_out(self):
        return self.terms[0].H_out

    @property
    def W_out(self):
        return self.terms[0].W_out

    @property
    def C_out(self):
        return self.terms[0].C_out

    @property
    def E_out(self):
        return self.H_out * self.W_out * self.C_out


def make_layer(terms, weights, bias, weight_scale: float, out_scale: float) -> Layer:
    """Quantise W -> round(weight_scale * W) and bias -> round(out_scale * bias)."""
    lay = Layer(terms=list(terms), weights=[np.asarray(w, dtype=np.float64) for w in weights],
                bias=None if bias is None else np.asarray(bias, dtype=np.float64))
    t0 = lay.terms[0]
    for t in lay.terms:
        assert (t.H_out, t.W_out, t.C_out) == (t0.H_out, t0.W_out, t0.C_out)
    lay.E_in = max(t.in_offset + t.H * t.W * t.C_in for t in lay.terms)
    lay.quantized = [quantize(w, weight_scale).reshape(w.shape) for w in lay.weights]
    if lay.bias is not None:
        lay.bias_q = quantize(lay.bias, out_scale)
    return lay


def output_taps(layer: Layer, o: int):
    """Input indices and quantised weights feeding output o, where
    o = (h' * W_out + w') * C_out + c (channels last)."""
    Wo, Co = layer.W_out, layer.C_out
    co = o % Co
    hw = o // Co
    ho, wo = hw // Wo, hw % Wo
    idx, wts = [], []
    for t, wq in zip(layer.terms, layer.quantized):
        for dh in range(t.kh):
            h = ho * t.stride - t.pad + dh
            if h < 0 or h >= t.H:
                continue
            for dw in range(t.kw):
                w = wo * t.stride - t.pad + dw
                if w < 0 or w >= t.W:
                    continue
                base = t.in_offset + (h * t.W + w) * t.C_in
                idx.extend(range(base, base + t.C_in))
                wts.extend(int(v) for v in wq[co, dh, dw, :])
    return np.array(idx, dtype=np.int64), np.array(wts, dtype=np.int64)


def dense_matrix(layer: Layer) -> np.ndarray:
    """The layer as an E' x E_in integer matrix (Toeplitz form of the conv,
    Sec. 5), as Python-int objects: the plain definition of f(x) = Ax."""
    A = np.zeros((layer.E_out, layer.E_in), dtype=object)
    for o in range(layer.E_out):
        idx, wts = output_taps(layer, o)
        for i, w in zip(idx, wts):
            A[o, i] += int(w)
    return A


def inverse_perm(perm) -> np.ndarray:
    perm = np.asarray(perm, dtype=np.int64)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size, dtype=np.int64)
    return inv


def extract(prm: Params, ct: np.ndarray, i: int, gamma: int = 0, power=None) -> np.ndarray:
    """Lemma 1 (Sec. 4.4 "Partial trace extraction") at t = 2: the RLWE row
    whose partial trace over K_gamma / K_0 holds coefficient i, with
    Omega_i^*-bar(X^d) = X^(-d i) / N.  gamma 0 (and 1, the same at t = 2
    since K_1 = K_0): N^-1 X^-i ct, and the full trace (degree N) returns
    m_i.  gamma 2: (N/2)^-1 (X^-i ct + X^-3i ct3), ct3 = RLWE_s(m(X^3)) the
    client's power (Sec. 4.3, j = 1, k in {0, 1}): Lemma 1's sum scaled by
    [K_2 : K_0] = 2, so that the server's trace over K / K_2 (degree N/2)
    cancels the scalar exactly and the packed value is 2 m_i, which the
    client halves after decryption (the paper removes this factor with
    M^-1 mod p in its torus encoding, which a fixed-point encoding cannot
    do without multiplying the fresh noise of ct3 by 2^-1 mod Q)."""
    inv = (lambda qi: pow(prm.n, -1, qi)) if gamma == 0 else (lambda qi: pow(prm.n // 2, -1, qi))

    def term(c, e):
        c = ct_monomial(prm, c, -e)
        for li, qi in enumerate(prm.q):
            c[:, li] = np.array([int(v) * inv(qi) % qi for v in c[:, li].ravel()],
                                dtype=np.uint64).reshape(c[:, li].shape)
        return c
    row = term(_u64(ct).reshape(2, prm.L, prm.n), i)
    if gamma == 2:
        row = ct_add(prm, row, term(_u64(power).reshape(2, prm.L, prm.n), 3 * i))
    return row


def client_power(prm: Params, m) -> np.ndarray:
    """The client's power for gamma = 2 at t = 2 (Sec. 4.3): m(X^3) of one
    chunk of N integer message coefficients, as integers."""
    m = np.asarray(m, dtype=np.int64)
    out = np.zeros(prm.n, dtype=object)
    for k, v in enumerate(m):
        e = 3 * k % (2 * prm.n)
        if e < prm.n:
            out[e] += int(v)
        else:
            out[e - prm.n] -= int(v)
    return np.array([int(v) for v in out], dtype=np.int64)


def linear_output(prm: Params, layer: Layer, cts: np.ndarray, o: int, sigma_prev=None,
                  powers: np.ndarray | None = None) -> np.ndarray:
    """RLWE row of output o before shuffling and packing:
    y_o = sum_i W[o,i] * (extracted row of input i), where input i sits at
    stream position sigma_prev^-1(i) (Sec. 4.4 "Unshuffle").  With the
    client's powers (gamma = 2, one per input ciphertext) the extracted row
    is (N/2)^-1 (X^-k ct_j + X^(-3k) ct3_j) (see extract): the taps count
    twice (weights 2 Wq against N^-1) and again at exponent 3k on ct3_j,
    where X^-e = -X^-(e - N) for N <= e < 2N."""
    cts = _u64(cts).reshape(-1, 2, prm.L, prm.n)
    idx, wts = output_taps(layer, o)
    if sigma_prev is None:
        pos = idx
    else:
        pos = inverse_perm(sigma_prev)[idx]
    pos = _i64(pos)
    wts = _i64(wts if powers is None else 2 * wts)
    q = _u64(prm.q)
    out = np.zeros((2, prm.L, prm.n), dtype=np.uint64)
    lib().or_linear_output(prm.n, prm.L, _p(q, _u64p), cts.shape[0], _p(cts, _u64p), pos.size,
                           _p(pos, _i64p), _p(wts, _i64p), _p(out, _u64p))
    if powers is not None:
        pw = _u64(powers).reshape(-1, 2, prm.L, prm.n)
        e = 3 * (pos % prm.n) % (2 * prm.n)
        pos3 = _i64((pos // prm.n) * prm.n + np.where(e < prm.n, e, e - prm.n))
        w3 = _i64(np.where(e < prm.n, wts, -wts))
        out3 = np.zeros_like(out)
        lib().or_linear_output(prm.n, prm.L, _p(q, _u64p), pw.shape[0], _p(pw, _u64p), pos3.size,
                               _p(pos3, _i64p), _p(w3, _i64p), _p(out3, _u64p))
        out = ct_add(prm, out, out3)
    return out


def add_bias(prm: Params, ct: np.ndarray, values, stride: int) -> np.ndarray:
    """b-part coefficient l*stride += values[l] (the affine part of f(x) = Ax + b)."""
    ct = _u64(ct).copy()
    for l, v in enumerate(values):
        for i, qi in enumerate(prm.q):
            ct[1, i, l * stride] = (int(ct[1, i, l * stride]) + int(v)) % qi
    return ct


def eval_linear_layer(prm: Params, layer: Layer, keys: dict, cts: np.ndarray,
                      sigma_prev=None, sigma_out=None, counter: Counter | None = None,
                      powers: np.ndarray | None = None) -> np.ndarray:
    """One server round (Sec. 4.4): for every output group g (n values per
    packed ciphertext, the same n for every group; the last group is padded
    with zero ciphertexts), leaf l = y_{sigma_out(g n + l)}, pack, add bias.
    With the client's powers (gamma = 2) the leaves use them and the packing
    skips the tau_3 level.  Returns [groups][2][L][N]."""
    gamma = 0 if powers is None else 2
    e_out = layer.E_out
    n = group_size(prm, e_out)
    groups = -(-e_out // n)
    perm = np.arange(e_out) if sigma_out is None else np.asarray(sigma_out, dtype=np.int64)
    out = []
    for g in range(groups):
        members = [int(perm[g * n + l]) for l in range(min(n, e_out - g * n))]
        leaves = [linear_output(prm, layer, cts, o, sigma_prev, powers) for o in members]
        ct = pack(prm, keys, leaves, counter, n=n, gamma=gamma)
        if layer.bias_q is not None:
            # at gamma = 2 the packed values carry [K_2 : K_0] = 2, the bias too
            co = np.array(members) % layer.C_out
            ct = add_bias(prm, ct, [(1 + (gamma == 2)) * int(layer.bias_q[c]) for c in co], prm.n // n)
        out.append(ct)
    return np.stack(out)


def read_outputs(prm: Params, layer: Layer, residues: np.ndarray, scale: float, gamma: int = 0) -> np.ndarray:
    """Client side (Sec. 4.5): read the packed positions l*N/n of each group
    and drop the padding; the result is in shuffled order sigma_out.  At
    gamma = 2 the packed values carry the factor [K_2 : K_0] = 2 (see extract)."""
    if gamma == 2:
        scale = 2 * scale
    e_out = layer.E_out
    n = group_size(prm, e_out)
    stride = prm.n // n
    vals = []
    for g in range(residues.shape[0]):
        cnt = min(n, e_out - g * n)
        sel = residues[g][:, [l * stride for l in range(cnt)]]
        vals.extend(decode(prm, sel, scale))
    return np.array(vals)
