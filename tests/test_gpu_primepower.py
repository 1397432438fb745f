"""Prime-power cyclotomic rings on the GPU (Sec. 2.1-2.3; Table 2's M = 3^7,
7^4, 5^5) against the exact prime-power oracle, residue by residue:
the length-M transform against direct evaluation at powers of omega, products
modulo Phi_M against the oracle's schoolbook product, automorphisms, and the
tower trace (full and partial) with its automorphism count."""
import numpy as np
import pytest
import torch

import paper_2509_01253_gb300 as sf
from oracle import primepower as pp

pytestmark = pytest.mark.gpu

# rings with a compile-time transform and, (3, 5) and (7, 3), rings on the generic one
CASES = [(3, 3, 2), (3, 4, 3), (5, 2, 2), (7, 2, 2), (5, 3, 1), (3, 7, 2), (7, 4, 1), (5, 5, 1), (3, 5, 2), (7, 3, 1)]


def _ring(t, alpha, L):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    r = sf.sf_pp_ring_create(t, alpha, L, 50, 0)
    return r, sf.sf_pp_ring_info(r, L)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def _digit_rev(j, t, alpha):
    r = 0
    for _ in range(alpha):
        r = r * t + j % t
        j //= t
    return r


def _rand(rng, mods, count, n):
    return np.stack([np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in mods]) for _ in range(count)])


@pytest.mark.parametrize("t,alpha,L", CASES)
def test_pp_ntt_is_evaluation_at_powers_of_omega(t, alpha, L):
    r, info = _ring(t, alpha, L)
    try:
        M, mods = info["M"], info["moduli"]
        for q in mods:
            assert q % M == 1 and q < 2 ** 50
        rng = np.random.default_rng(7 * t + alpha)
        a = _rand(rng, mods, 2, M)
        A = torch.zeros((2, L, M), dtype=torch.int64, device="cuda")
        sf.sf_pp_ntt(r, _dev(a), A, 2, False)
        ha = _host(A)
        # omega from the transform of X: out[j] = omega^rev(j), out[1] = omega^rev(1) = omega^(M/t)
        x = np.zeros((1, L, M), dtype=np.uint64)
        x[0, :, 1] = 1
        X = _dev(x)
        sf.sf_pp_ntt(r, X, X, 1, False)
        hx = _host(X)[0]
        for i, q in enumerate(mods):
            w = int(hx[i, _digit_rev(1, t, alpha)])           # omega^1 sits at slot rev(1)
            assert pow(w, M, q) == 1 and pow(w, M // t, q) != 1  # a primitive M-th root
            for j in rng.choice(M, 12, replace=False):
                k = _digit_rev(int(j), t, alpha)
                wk = pow(w, k, q)
                want = 0
                for c in reversed(a[1, i].tolist()):           # Horner: a(omega^k)
                    want = (want * wk + c) % q
                assert int(ha[1, i, j]) == want, (i, j)
        back = torch.zeros_like(A)
        sf.sf_pp_ntt(r, A, back, 2, True)
        assert (_host(back) == a).all()
        sf.sf_pp_ntt(r, A, A, 2, True)                        # in place
        assert (_host(A) == a).all()
        with pytest.raises(sf.SafhireError):
            sf.sf_pp_ntt(r, A, A, 0, False)
    finally:
        sf.sf_pp_ring_destroy(r)


@pytest.mark.parametrize("t,alpha,L", CASES)
def test_pp_mul_and_automorphism_match_oracle(t, alpha, L):
    r, info = _ring(t, alpha, L)
    try:
        R = pp.Ring(t, alpha)
        N, mods = info["N"], info["moduli"]
        assert N == R.N
        rng = np.random.default_rng(11 * t + alpha)
        a = _rand(rng, mods, 2, N)
        b = _rand(rng, mods, 2, N)
        out = torch.zeros((2, L, N), dtype=torch.int64, device="cuda")
        sf.sf_pp_mul(r, _dev(a), _dev(b), out, 2)
        got = _host(out)
        # the oracle's exact product in Z[X]/Phi_M, reduced mod q (a ring map);
        # one limb at the largest rings, where the schoolbook product is slow
        limbs = [(c, i) for c in range(2) for i in range(L)] if N <= 600 else [(1, L - 1)]
        for c, i in limbs:
            q = mods[i]
            want = R.mod(R.mul([int(v) for v in a[c, i]], [int(v) for v in b[c, i]]), q)
            assert [int(v) for v in got[c, i]] == want, (c, i)
        units = [d for d in (2, t + 1, R.M - 1, 5 * t + 2) if d % t and d < R.M]
        for d in units:
            sf.sf_pp_automorphism(r, _dev(a), out, 2, d)
            got = _host(out)
            for c, i in limbs:
                want = R.mod(R.automorphism([int(v) for v in a[c, i]], d), mods[i])
                assert [int(v) for v in got[c, i]] == want, (d, c, i)
        with pytest.raises(sf.SafhireError):
            sf.sf_pp_automorphism(r, _dev(a), out, 2, t)          # not coprime to M
    finally:
        sf.sf_pp_ring_destroy(r)


@pytest.mark.parametrize("t,alpha,L", [(3, 3, 2), (3, 4, 1), (5, 2, 2), (7, 2, 1), (5, 3, 1), (3, 7, 1)])
def test_pp_trace_tower_matches_oracle(t, alpha, L):
    r, info = _ring(t, alpha, L)
    try:
        R = pp.Ring(t, alpha)
        N, mods = info["N"], info["moduli"]
        rng = np.random.default_rng(13 * t + alpha)
        a = _rand(rng, mods, 1, N)
        out = torch.zeros((1, L, N), dtype=torch.int64, device="cuda")
        for gamma in range(0, alpha + 1):
            n_auto = sf.sf_pp_trace(r, _dev(a), out, 1, gamma)
            assert n_auto == R.tower_ks_count(gamma), gamma
            got = _host(out)
            for i, q in enumerate(mods):
                x = [int(v) for v in a[0, i]]
                want = R.mod(R.tower_trace(x, gamma), q)
                assert [int(v) for v in got[0, i]] == want, (gamma, i)
                if N <= 200:   # the definitions: sum over the Galois group
                    ref = R.partial_trace(x, gamma) if gamma >= 1 else R.trace(x)
                    assert want == R.mod(ref, q), (gamma, i)
    finally:
        sf.sf_pp_ring_destroy(r)


def test_pp_ring_rejects_bad_parameters():
    for args in ((2, 5, 1, 50), (9, 2, 1, 50), (11, 2, 1, 50), (3, 1, 1, 50), (3, 8, 1, 50), (3, 3, 0, 50),
                 (3, 3, 1, 62)):
        with pytest.raises(sf.SafhireError):
            sf.sf_pp_ring_create(*args, 0)


# --------------------------------------------------------------- RLWE ------

def _i64(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.int64))).cuda()


def _ct_lists(h, L, N):
    """uint64[2][L][N] -> the oracle's ([a limbs], [b limbs]) of Python ints."""
    return ([[int(v) for v in h[0, j]] for j in range(L)], [[int(v) for v in h[1, j]] for j in range(L)])


def _setup_rlwe(t, alpha, L, seed):
    r, info = _ring(t, alpha, L)
    R = pp.Ring(t, alpha)
    E = pp.RnsRlwe(R, info["moduli"])
    rng = np.random.default_rng(seed)
    N = R.N
    s = rng.integers(-1, 2, N)
    return r, info, R, E, rng, N, s


def _key(r, E, R, rng, s, h, L, N, noise=True):
    ka = np.stack([_rand(rng, E.q, 1, N)[0] for _ in range(L)])           # [L digits][L limbs][N]
    ek = rng.integers(-3, 4, (L, N)) if noise else np.zeros((L, N), dtype=np.int64)
    d_ka, d_kb = _dev(ka), torch.zeros((L, L, N), dtype=torch.int64, device="cuda")
    sf.sf_pp_ksk(r, _i64(s), h, d_ka, _i64(ek), d_kb)
    return ka, ek, d_ka, d_kb


@pytest.mark.parametrize("t,alpha,L,h", [(3, 3, 2, 10), (3, 4, 3, 28), (5, 2, 2, 6), (7, 2, 2, 8)])
def test_pp_rlwe_encrypt_keyswitch_match_oracle(t, alpha, L, h):
    """Encryption, decryption, the key for tau_h and the key switch, every
    residue against the oracle's RnsRlwe on the same s, masks and noise."""
    r, info, R, E, rng, N, s = _setup_rlwe(t, alpha, L, 101 + t * alpha)
    try:
        count = 2
        a = _rand(rng, E.q, count, N)
        m = rng.integers(-2 ** 40, 2 ** 40, (count, N))
        e = rng.integers(-8, 9, (count, N))
        ct = torch.zeros((count, 2, L, N), dtype=torch.int64, device="cuda")
        sf.sf_pp_encrypt(r, _i64(s), _dev(a), _i64(m), _i64(e), ct, count)
        hct = _host(ct)
        sl = [int(v) for v in s]
        for c in range(count):
            want = E.encrypt(sl, [[int(v) for v in a[c, j]] for j in range(L)], m[c].tolist(), e[c].tolist())
            assert _ct_lists(hct[c], L, N) == want, c
        dec = torch.zeros((count, L, N), dtype=torch.int64, device="cuda")
        sf.sf_pp_decrypt(r, _i64(s), ct, dec, count)
        hd = _host(dec)
        assert E.centered([[int(v) for v in hd[0, j]] for j in range(L)]) == (m[0] + e[0]).tolist()
        ka, ek, d_ka, d_kb = _key(r, E, R, rng, s, h, L, N)
        kb_want = E.ksk(sl, h, [[[int(v) for v in ka[i, j]] for j in range(L)] for i in range(L)], ek.tolist())
        hkb = _host(d_kb)
        assert [[[int(v) for v in hkb[i, j]] for j in range(L)] for i in range(L)] == kb_want
        out = torch.zeros_like(ct)
        sf.sf_pp_keyswitch(r, ct, out, count, h, d_ka, d_kb)
        hout = _host(out)
        ka_l = [[[int(v) for v in ka[i, j]] for j in range(L)] for i in range(L)]
        for c in range(count):
            want = E.keyswitch(_ct_lists(hct[c], L, N), h, ka_l, kb_want)
            assert _ct_lists(hout[c], L, N) == want, c
    finally:
        sf.sf_pp_ring_destroy(r)


@pytest.mark.parametrize("t,alpha,L", [(3, 3, 2), (5, 2, 2), (7, 2, 2)])
def test_pp_hom_trace_matches_oracle(t, alpha, L):
    """The homomorphic tower trace at every gamma, residue by residue against
    the oracle with noisy keys, and its key-switch count."""
    r, info, R, E, rng, N, s = _setup_rlwe(t, alpha, L, 211 + t * alpha)
    try:
        a = _rand(rng, E.q, 1, N)
        m = rng.integers(-2 ** 30, 2 ** 30, (1, N))
        e = rng.integers(-8, 9, (1, N))
        ct = torch.zeros((1, 2, L, N), dtype=torch.int64, device="cuda")
        sf.sf_pp_encrypt(r, _i64(s), _dev(a), _i64(m), _i64(e), ct, 1)
        hct = _host(ct)
        sl = [int(v) for v in s]
        keys_dev, keys_or = {}, {}
        for gamma in range(0, alpha + 1):
            for h, _ in R.tower_steps(gamma):
                if h not in keys_dev:
                    ka, ek, d_ka, d_kb = _key(r, E, R, rng, s, h, L, N)
                    ka_l = [[[int(v) for v in ka[i, j]] for j in range(L)] for i in range(L)]
                    keys_dev[h] = (d_ka, d_kb)
                    keys_or[h] = (ka_l, E.ksk(sl, h, ka_l, ek.tolist()))
        out = torch.zeros_like(ct)
        for gamma in range(0, alpha + 1):
            n_ks = sf.sf_pp_hom_trace(r, ct, out, 1, gamma, keys_dev)
            assert n_ks == R.tower_ks_count(gamma)
            want = E.hom_trace(_ct_lists(hct[0], L, N), gamma, keys_or)
            assert _ct_lists(_host(out)[0], L, N) == want, gamma
        with pytest.raises(sf.SafhireError):
            sf.sf_pp_hom_trace(r, ct, out, 1, 0, {})            # no keys
    finally:
        sf.sf_pp_ring_destroy(r)


def test_pp_hom_trace_largest_ring_decrypts_to_the_trace():
    """M = 3^7 (N = 1458, Table 2's first ring), two 30-bit limbs: with
    noiseless keys the homomorphic trace at every gamma decrypts exactly to
    Tr_{K/K_gamma}(m + e) (the oracle's plaintext tower trace), and one key
    switch with a noisy key matches the oracle residue by residue."""
    t, alpha, L = 3, 7, 2
    r, info, R, E, rng, N, s = _setup_rlwe(t, alpha, L, 307)
    try:
        a = _rand(rng, E.q, 1, N)
        m = rng.integers(-2 ** 20, 2 ** 20, (1, N))
        e = rng.integers(-8, 9, (1, N))
        ct = torch.zeros((1, 2, L, N), dtype=torch.int64, device="cuda")
        sf.sf_pp_encrypt(r, _i64(s), _dev(a), _i64(m), _i64(e), ct, 1)
        keys = {}
        for h, _ in R.tower_steps(0):
            _, _, d_ka, d_kb = _key(r, E, R, rng, s, h, L, N, noise=False)
            keys[h] = (d_ka, d_kb)
        me = (m[0] + e[0]).tolist()
        out = torch.zeros_like(ct)
        dec = torch.zeros((1, L, N), dtype=torch.int64, device="cuda")
        for gamma in (0, 1, 3, 6):
            sf.sf_pp_hom_trace(r, ct, out, 1, gamma, keys)
            sf.sf_pp_decrypt(r, _i64(s), out, dec, 1)
            hd = _host(dec)
            got = E.centered([[int(v) for v in hd[0, j]] for j in range(L)])
            assert got == R.tower_trace(me, gamma), gamma
        h = R.tower_steps(0)[0][0]
        ka, ek, d_ka, d_kb = _key(r, E, R, rng, s, h, L, N)
        sl = [int(v) for v in s]
        ka_l = [[[int(v) for v in ka[i, j]] for j in range(L)] for i in range(L)]
        sf.sf_pp_keyswitch(r, ct, out, 1, h, d_ka, d_kb)
        want = E.keyswitch(_ct_lists(_host(ct)[0], L, N), h, ka_l, E.ksk(sl, h, ka_l, ek.tolist()))
        assert _ct_lists(_host(out)[0], L, N) == want
    finally:
        sf.sf_pp_ring_destroy(r)
