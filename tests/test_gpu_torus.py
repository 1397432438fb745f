"""The paper's torus scheme on the GPU (RLWE over T_q, q = 2^53, Sec. 2.1;
the gadget key switching of Sec. 2.2 / Sec. 4.2 with Table 2's (D, l); the
homomorphic tower trace of Sec. 2.3) against the oracle's TorusRlwe, word by
word: gadget digits, ciphertexts, phases, keys, key switches and traces, on
the small test rings (compiled and generic transforms) and at Table 2's
full sizes, including one launch of 4096 ciphertexts checked on samples."""
import numpy as np
import pytest
import torch

import paper_2509_01253_gb300 as sf
from oracle import primepower as pp

pytestmark = pytest.mark.gpu

Q = 2 ** 53
# Table 2's rings and gadgets (t, alpha, D, l)
TABLE2 = [(3, 7, 512, 3), (7, 4, 2 ** 12, 3), (7, 4, 2 ** 16, 2), (5, 5, 310, 5), (5, 5, 310, 4)]
# compiled rings, and (3, 5), (7, 3) on the generic transform
SMALL = [(3, 3, 512, 3), (5, 2, 310, 5), (7, 2, 2 ** 16, 2), (3, 4, 2 ** 12, 3), (5, 3, 3, 8), (3, 5, 512, 3),
         (7, 3, 310, 4)]


def _ring(t, alpha, D, l):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    r = sf.sf_tq_ring_create(t, alpha, D, l, 0)
    return r, sf.sf_tq_ring_info(r)


def _dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a.astype(np.int64, copy=False)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def _torus(rng, *shape):
    return rng.integers(0, Q, shape, dtype=np.uint64)


def _L(x):
    return [int(v) for v in x]


class _Setup:
    def __init__(self, t, alpha, D, l, seed):
        self.r, self.info = _ring(t, alpha, D, l)
        self.R = pp.Ring(t, alpha)
        self.T = pp.TorusRlwe(self.R, D, l)
        self.rng = np.random.default_rng(seed)
        self.N, self.l = self.R.N, l
        self.s = self.rng.integers(-1, 2, self.N)
        self.d_s = _dev(self.s)

    def encrypt(self, count, noise=2 ** 17):
        a = _torus(self.rng, count, self.N)
        m = _torus(self.rng, count, self.N)
        e = self.rng.integers(-noise, noise + 1, (count, self.N))
        ct = torch.zeros((count, 2, self.N), dtype=torch.int64, device="cuda")
        sf.sf_tq_encrypt(self.r, self.d_s, _dev(a), _dev(m), _dev(e), ct, count)
        return a, m, e, ct

    def key(self, h, noise=2 ** 17):
        ka = _torus(self.rng, self.l, self.N)
        ek = self.rng.integers(-noise, noise + 1, (self.l, self.N)) if noise else np.zeros((self.l, self.N), np.int64)
        d_ka, d_kb = _dev(ka), torch.zeros((self.l, self.N), dtype=torch.int64, device="cuda")
        sf.sf_tq_ksk(self.r, self.d_s, h, d_ka, _dev(ek), d_kb)
        d_key = torch.zeros(self.info["key_words"], dtype=torch.int64, device="cuda")
        sf.sf_tq_key_prepare(self.r, d_ka, d_kb, d_key)
        ka_l = [_L(row) for row in ka]
        kb_want = self.T.ksk(_L(self.s), h, ka_l, ek.tolist())
        return d_kb, d_key, ka_l, kb_want

    def ct_lists(self, hct):
        return (_L(hct[0]), _L(hct[1]))


def test_tq_ring_info():
    for t, alpha, D, l in TABLE2:
        r, info = _ring(t, alpha, D, l)
        try:
            M = t ** alpha
            assert info["M"] == M and info["N"] == M - M // t
            assert info["key_words"] == 8 * l * M
            for p in info["primes"]:
                assert p % M == 1 and 2 ** 49 < p < 2 ** 50
        finally:
            sf.sf_tq_ring_destroy(r)


@pytest.mark.parametrize("t,alpha,D,l", SMALL + [(5, 5, 310, 5), (7, 4, 2 ** 16, 2), (3, 3, 2, 8)])
def test_tq_decompose_matches_oracle(t, alpha, D, l):
    S = _Setup(t, alpha, D, l, 17 * t + l)
    try:
        count = 3
        x = _torus(S.rng, count, S.N)
        x[0, :6] = np.array([0, 1, Q - 1, Q // 2, Q // 2 - 1, Q // D ** l * 3], dtype=np.uint64)
        x[1, 0] = np.uint64(2 ** 64 - 1)                     # read modulo 2^53
        dig = torch.zeros((count, l, S.N), dtype=torch.int32, device="cuda")
        sf.sf_tq_decompose(S.r, _dev(x), dig, count)
        torch.cuda.synchronize()
        hd = dig.cpu().numpy()
        for c in range(count):
            want = S.T.decompose([int(v) % Q for v in x[c]])
            assert [_L(hd[c, i]) for i in range(l)] == want, c
    finally:
        sf.sf_tq_ring_destroy(S.r)


@pytest.mark.parametrize("t,alpha,D,l", SMALL)
def test_tq_encrypt_keyswitch_match_oracle(t, alpha, D, l):
    """Encryption, the phase, the key for tau_h and the key switch, every
    word against the oracle on the same secret, masks and noise."""
    S = _Setup(t, alpha, D, l, 101 + t * alpha + l)
    try:
        count = 3
        a, m, e, ct = S.encrypt(count)
        hct = _host(ct)
        sl = _L(S.s)
        for c in range(count):
            assert S.ct_lists(hct[c]) == S.T.encrypt(sl, _L(a[c]), _L(m[c]), e[c].tolist()), c
        ph = torch.zeros((count, S.N), dtype=torch.int64, device="cuda")
        sf.sf_tq_decrypt(S.r, S.d_s, ct, ph, count)
        hph = _host(ph)
        for c in range(count):
            assert _L(hph[c]) == [(int(x) + int(y)) % Q for x, y in zip(m[c], e[c])]
        for h in S.R.units()[1:4]:
            d_kb, d_key, ka_l, kb_want = S.key(h)
            assert [_L(row) for row in _host(d_kb)] == kb_want
            out = torch.zeros_like(ct)
            sf.sf_tq_keyswitch(S.r, ct, out, count, h, d_key)
            hout = _host(out)
            for c in range(count):
                assert S.ct_lists(hout[c]) == S.T.keyswitch(S.ct_lists(hct[c]), h, ka_l, kb_want), (h, c)
        with pytest.raises(sf.SafhireError):
            sf.sf_tq_keyswitch(S.r, ct, ct, count, h, d_key)        # in place
        with pytest.raises(sf.SafhireError):
            sf.sf_tq_keyswitch(S.r, ct, out, count, t, d_key)       # not a unit
    finally:
        sf.sf_tq_ring_destroy(S.r)


@pytest.mark.parametrize("t,alpha,D,l", [(3, 3, 512, 3), (5, 2, 310, 5), (7, 2, 2 ** 12, 3), (3, 5, 2 ** 16, 2)])
def test_tq_hom_trace_matches_oracle(t, alpha, D, l):
    """The homomorphic tower trace at every gamma with noisy keys, word by
    word against the oracle, and its key-switch count."""
    S = _Setup(t, alpha, D, l, 211 + t * alpha)
    try:
        _, _, _, ct = S.encrypt(2)
        hct = _host(ct)
        keys_dev, keys_or = {}, {}
        for gamma in range(alpha + 1):
            for h, _ in S.R.tower_steps(gamma):
                if h not in keys_dev:
                    _, d_key, ka_l, kb_want = S.key(h)
                    keys_dev[h], keys_or[h] = d_key, (ka_l, kb_want)
        out = torch.zeros_like(ct)
        for gamma in range(alpha + 1):
            assert sf.sf_tq_hom_trace(S.r, ct, out, 2, gamma, keys_dev) == S.R.tower_ks_count(gamma)
            hout = _host(out)
            for c in range(2):
                assert S.ct_lists(hout[c]) == S.T.hom_trace(S.ct_lists(hct[c]), gamma, keys_or), (gamma, c)
        with pytest.raises(sf.SafhireError):
            sf.sf_tq_hom_trace(S.r, ct, out, 2, 0, {})               # no keys
        with pytest.raises(sf.SafhireError):
            sf.sf_tq_hom_trace(S.r, ct, ct, 2, 0, keys_dev)          # in place
    finally:
        sf.sf_tq_ring_destroy(S.r)


@pytest.mark.parametrize("t,alpha,D,l", TABLE2)
def test_tq_table2_keyswitch_matches_oracle(t, alpha, D, l):
    """Table 2's rings and gadgets at full size: keys and one key switch of two
    ciphertexts, word by word."""
    S = _Setup(t, alpha, D, l, 307 + D + l)
    try:
        _, _, _, ct = S.encrypt(2)
        hct = _host(ct)
        h = S.R.tower_steps(0)[0][0]
        d_kb, d_key, ka_l, kb_want = S.key(h)
        assert [_L(row) for row in _host(d_kb)] == kb_want
        out = torch.zeros_like(ct)
        sf.sf_tq_keyswitch(S.r, ct, out, 2, h, d_key)
        hout = _host(out)
        for c in range(2):
            assert S.ct_lists(hout[c]) == S.T.keyswitch(S.ct_lists(hct[c]), h, ka_l, kb_want), c
    finally:
        sf.sf_tq_ring_destroy(S.r)


def test_tq_table2_batch_launch_sampled():
    """M = 5^5, (D, l) = (310, 5): one key-switch launch over 4096 ciphertexts
    (the size the bench times), sampled ciphertexts against the oracle."""
    S = _Setup(5, 5, 310, 5, 401)
    try:
        count = 4096
        _, _, _, ct = S.encrypt(count)
        h = S.R.tower_steps(0)[0][0]
        _, d_key, ka_l, kb_want = S.key(h)
        out = torch.zeros_like(ct)
        sf.sf_tq_keyswitch(S.r, ct, out, count, h, d_key)
        hct, hout = _host(ct), _host(out)
        for c in (0, 1, 2047, 4095):
            assert S.ct_lists(hout[c]) == S.T.keyswitch(S.ct_lists(hct[c]), h, ka_l, kb_want), c
    finally:
        sf.sf_tq_ring_destroy(S.r)


def test_tq_table2_trace_decodes_to_the_trace():
    """M = 3^7 with (512, 3) and Delta = 2^-36 (Table 2, b = 8): the full
    homomorphic trace of an encrypted 8-bit message matches the oracle word by
    word and decodes to Tr(mu) mod 2^8."""
    S = _Setup(3, 7, 512, 3, 503)
    try:
        b, sigma = 8, 2 ** 17
        mu = S.rng.integers(0, 2 ** b, S.N)
        m = np.array(S.T.encode(mu.tolist(), b), dtype=np.uint64)[None]
        a = _torus(S.rng, 1, S.N)
        e = np.rint(S.rng.normal(0.0, sigma, (1, S.N))).astype(np.int64)
        ct = torch.zeros((1, 2, S.N), dtype=torch.int64, device="cuda")
        sf.sf_tq_encrypt(S.r, S.d_s, _dev(a), _dev(m), _dev(e), ct, 1)
        keys_dev, keys_or = {}, {}
        for h, _ in S.R.tower_steps(0):
            _, d_key, ka_l, kb_want = S.key(h, noise=sigma)
            keys_dev[h], keys_or[h] = d_key, (ka_l, kb_want)
        out = torch.zeros_like(ct)
        sf.sf_tq_hom_trace(S.r, ct, out, 1, 0, keys_dev)
        want = S.T.hom_trace(S.ct_lists(_host(ct)[0]), 0, keys_or)
        assert S.ct_lists(_host(out)[0]) == want
        ph = torch.zeros((1, S.N), dtype=torch.int64, device="cuda")
        sf.sf_tq_decrypt(S.r, S.d_s, out, ph, 1)
        assert S.T.decode(_L(_host(ph)[0]), b) == [v % 2 ** b for v in S.R.tower_trace(mu.tolist(), 0)]
    finally:
        sf.sf_tq_ring_destroy(S.r)


def test_tq_edge_cases():
    """Input words are read modulo 2^53 (high bits set change nothing), a single
    ciphertext, gamma = alpha (no automorphism: the trace is the input, zero
    key switches), a key prepared twice gives the same words, and a negative
    automorphism index is taken modulo M."""
    S = _Setup(3, 3, 512, 3, 601)
    try:
        _, _, _, ct = S.encrypt(1)
        hct = _host(ct)
        h = 10
        d_kb, d_key, ka_l, kb_want = S.key(h)
        ref = S.T.keyswitch(S.ct_lists(hct[0]), h, ka_l, kb_want)
        dirty = hct.copy()
        dirty |= np.uint64(0x7FF) << np.uint64(53)               # bits 53..63 set
        out = torch.zeros_like(ct)
        sf.sf_tq_keyswitch(S.r, _dev(dirty), out, 1, h, d_key)
        assert S.ct_lists(_host(out)[0]) == ref
        sf.sf_tq_keyswitch(S.r, ct, out, 1, h - S.R.M, d_key)     # h - M = h (mod M)
        assert S.ct_lists(_host(out)[0]) == ref
        again = torch.zeros_like(d_key)
        sf.sf_tq_key_prepare(S.r, _dev(np.array(ka_l, dtype=np.uint64)), d_kb, again)
        assert torch.equal(again, d_key)
        tr = torch.zeros_like(ct)
        assert sf.sf_tq_hom_trace(S.r, ct, tr, 1, S.R.alpha, {}) == 0
        assert torch.equal(tr, ct)
    finally:
        sf.sf_tq_ring_destroy(S.r)
