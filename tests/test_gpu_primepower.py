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
