"""Pins of the prime-power ring oracle (oracle/primepower.py; the paper's
M = t^alpha rings, Sec. 2.1-2.4) to facts that do not come from it:
evaluation at primitive M-th roots of unity modulo a prime p = 1 (mod M)
(a ring homomorphism of K onto Z_p for every unit exponent), Ramanujan's
closed form of the trace of a monomial, the trace as a sum of all
evaluations, the definition of the partial traces, and the dual basis at
t = 2 (X^i / N)."""
import math
import random

import pytest
import sympy

from oracle import primepower as pp

RINGS = [(3, 2), (3, 3), (5, 2), (7, 2), (13, 1)]


def _root(M):
    """A prime p = 1 (mod M) and a primitive M-th root of unity mod p (sympy)."""
    p = M + 1
    while not sympy.isprime(p):
        p += M
    g = sympy.primitive_root(p)
    return p, pow(g, (p - 1) // M, p)


def _ev(a, x, p):
    return sum(int(c) * pow(x, i, p) for i, c in enumerate(a)) % p


@pytest.mark.parametrize("t,alpha", RINGS)
def test_product_and_automorphisms_by_evaluation(t, alpha):
    """At every primitive M-th root w^k (gcd(k, M) = 1) modulo p: the product
    evaluates to the product of evaluations, tau_d(a) evaluates to a at w^(k d),
    Phi_M vanishes, and tau_a tau_b = tau_(a b mod M)."""
    R = pp.Ring(t, alpha)
    p, w = _root(R.M)
    rng = random.Random(t * 100 + alpha)
    a = [rng.randint(-10 ** 6, 10 ** 6) for _ in range(R.N)]
    b = [rng.randint(-10 ** 6, 10 ** 6) for _ in range(R.N)]
    ab = R.mul(a, b)
    phi = [1 if e % R.m == 0 else 0 for e in range(R.M - R.m + 1)]
    assert R.reduce(phi) == [0] * R.N
    units = R.units()
    assert len(units) == R.N == sympy.totient(R.M)
    for k in units:
        x = pow(w, k, p)
        assert _ev(ab, x, p) == _ev(a, x, p) * _ev(b, x, p) % p
        for d in units[:5]:
            assert _ev(R.automorphism(a, d), x, p) == _ev(a, pow(w, k * d, p), p)
    d1, d2 = units[1], units[-2]
    assert R.automorphism(R.automorphism(a, d1), d2) == R.automorphism(a, d1 * d2 % R.M)


@pytest.mark.parametrize("t,alpha", RINGS)
def test_trace_of_monomials_is_a_ramanujan_sum(t, alpha):
    """Tr(X^j) = phi(M) if M | j, -M/t if M/t | j but M does not, 0 otherwise
    (the Ramanujan sum c_M(j) of a prime power)."""
    R = pp.Ring(t, alpha)
    for j in range(2 * R.M):
        want = R.N if j % R.M == 0 else (-R.m if j % R.m == 0 else 0)
        tr = R.trace(R.monomial(j))
        assert tr == [want] + [0] * (R.N - 1), j


@pytest.mark.parametrize("t,alpha", [(3, 3), (5, 2), (7, 2), (13, 1), (3, 4)])
def test_tower_trace_equals_trace_with_the_paper_count(t, alpha):
    """Sec. 2.3: the tower evaluation equals the trace by definition (a sum of
    N automorphisms; also the sum of the N evaluations at the primitive roots)
    with (alpha - 1)(t - 1) + sum_{l in omega(t - 1)} (l - 1) automorphisms;
    stopping at gamma gives the partial trace over K / K_gamma with
    (alpha - gamma)(t - 1)."""
    R = pp.Ring(t, alpha)
    p, w = _root(R.M)
    rng = random.Random(7 * t + alpha)
    a = [rng.randint(-1000, 1000) for _ in range(R.N)]
    c = [0]
    tr = R.tower_trace(a, 0, c)
    assert tr == R.trace(a)
    assert tr[0] % p == sum(_ev(a, pow(w, k, p), p) for k in R.units()) % p
    omega = sympy.factorint(t - 1)
    assert c[0] == (alpha - 1) * (t - 1) + sum((l - 1) * e for l, e in omega.items())
    for gamma in range(1, alpha + 1):
        c = [0]
        assert R.tower_trace(a, gamma, c) == R.partial_trace(a, gamma)
        assert c[0] == (alpha - gamma) * (t - 1) == R.tower_ks_count(gamma)


def test_dual_basis_at_t2_is_scaled_monomials():
    """At t = 2 the dual basis of the power basis is Omega_i^* = X^i / N."""
    R = pp.Ring(2, 4)
    for i, om in enumerate(R.dual_basis()):
        assert om == [pp.Fraction(int(k == i), R.N) for k in range(R.N)], i


@pytest.mark.parametrize("t,alpha", [(3, 2), (3, 3), (5, 2)])
def test_dual_basis_reads_coefficients(t, alpha):
    """Coefficient i of m is Tr(m Omega_i^*-bar) (Sec. 4.4), for random m."""
    R = pp.Ring(t, alpha)
    om = R.dual_basis()
    rng = random.Random(3)
    m = [rng.randint(-99, 99) for _ in range(R.N)]
    for i in range(R.N):
        tr = R.trace(R.mul(m, R.conj(om[i])))
        assert tr[0] == m[i] and all(v == 0 for v in tr[1:]), i


@pytest.mark.parametrize("t,alpha,gamma", [(3, 2, 1), (3, 3, 1), (3, 3, 2), (5, 2, 1), (5, 2, 2), (7, 2, 2)])
def test_lemma1_partial_trace_rows(t, alpha, gamma):
    """Lemma 1: the extracted row sum_{j, k} P(X^(k(jt+1))) Omega_i^*-bar(X^(k(jt+1)))
    (j < t at gamma = 2, j = 0 at gamma = 1; k = 1 .. t-1) is the partial trace
    over K_gamma / K_0 of P Omega_i^*-bar: the server's remaining trace over
    K / K_gamma (tower levels above gamma) maps it to exactly coefficient i."""
    R = pp.Ring(t, alpha)
    om = R.dual_basis()
    rng = random.Random(11 * t + gamma)
    P = [rng.randint(-50, 50) for _ in range(R.N)]
    js = range(t) if gamma == 2 else [0]
    reps = [k * (j * t + 1) % R.M for j in js for k in range(1, t)]
    assert len(set(r % t ** gamma for r in reps)) == (t - 1) * t ** (gamma - 1)   # one per coset of Gal(K / K_gamma)
    for i in range(0, R.N, max(1, R.N // 6)):
        obar = R.conj(om[i])
        row = [0] * R.N
        for d in reps:
            row = R.add(row, R.mul(R.automorphism(P, d), R.automorphism(obar, d)))
        out = R.tower_trace(row, gamma)
        assert out[0] == P[i] and all(v == 0 for v in out[1:]), i


# ---------------------------------------------------------------- RLWE ----

def _is_prime(n: int) -> bool:
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def _primes_1_mod(M: int, bits: int, count: int) -> list:
    out, k = [], ((1 << bits) - 2) // M
    while len(out) < count:
        if _is_prime(k * M + 1):
            out.append(k * M + 1)
        k -= 1
    return out


def _rlwe_setup(t, alpha, L, seed):
    R = pp.Ring(t, alpha)
    E = pp.RnsRlwe(R, _primes_1_mod(R.M, 30, L))
    rng = random.Random(seed)
    s = [rng.choice((-1, 0, 1)) for _ in range(R.N)]
    return R, E, rng, s


@pytest.mark.parametrize("t,alpha", [(3, 2), (3, 3), (5, 2), (7, 2)])
def test_rlwe_encrypt_decrypt_round_trip(t, alpha):
    """b - a s = m + e exactly (CRT of the limbs, centered)."""
    R, E, rng, s = _rlwe_setup(t, alpha, 3, 5 + t)
    m = [rng.randrange(-2 ** 40, 2 ** 40) for _ in range(R.N)]
    e = [rng.randrange(-8, 9) for _ in range(R.N)]
    a = [[rng.randrange(q) for _ in range(R.N)] for q in E.q]
    ct = E.encrypt(s, a, m, e)
    assert E.centered(E.decrypt(s, ct)) == [x + y for x, y in zip(m, e)]


@pytest.mark.parametrize("t,alpha,h", [(3, 2, 4), (3, 3, 10), (5, 2, 6), (7, 2, 3)])
def test_rlwe_keyswitch_is_the_automorphism(t, alpha, h):
    """With noiseless keys the key-switched tau_h(ct) decrypts to exactly
    tau_h(m + e); with noisy keys the extra term is -sum_i d_i e_i, bounded
    by sum_i q_i ||e_i||_1 times the ring's expansion."""
    R, E, rng, s = _rlwe_setup(t, alpha, 2, 17 + h)
    m = [rng.randrange(-2 ** 30, 2 ** 30) for _ in range(R.N)]
    e = [rng.randrange(-8, 9) for _ in range(R.N)]
    a = [[rng.randrange(q) for _ in range(R.N)] for q in E.q]
    ct = E.encrypt(s, a, m, e)
    ka = [[[rng.randrange(q) for _ in range(R.N)] for q in E.q] for _ in E.q]
    zero = [[0] * R.N for _ in E.q]
    kb = E.ksk(s, h, ka, zero)
    out = E.keyswitch(ct, h, ka, kb)
    want = R.automorphism([x + y for x, y in zip(m, e)], h)
    assert E.centered(E.decrypt(s, out)) == want
    ek = [[rng.randrange(-4, 5) for _ in range(R.N)] for _ in E.q]
    out = E.keyswitch(ct, h, ka, E.ksk(s, h, ka, ek))
    diff = [x - y for x, y in zip(E.centered(E.decrypt(s, out)), want)]
    bound = sum(q * sum(abs(v) for v in ek[i]) for i, q in enumerate(E.q)) * (R.t - 1)
    assert any(diff) and max(abs(v) for v in diff) <= bound


@pytest.mark.parametrize("t,alpha", [(3, 2), (3, 3), (5, 2), (7, 2)])
def test_rlwe_hom_trace_is_the_trace(t, alpha):
    """With noiseless keys the homomorphic tower trace decrypts to exactly
    Tr_{K/K_gamma}(m + e) by definition (the sum over Gal(K/K_gamma)), using
    (alpha - max(gamma,1))(t-1) (+ the K_1/K_0 steps) key switches."""
    R, E, rng, s = _rlwe_setup(t, alpha, 2, 31 + t)
    m = [rng.randrange(-2 ** 20, 2 ** 20) for _ in range(R.N)]
    e = [rng.randrange(-8, 9) for _ in range(R.N)]
    a = [[rng.randrange(q) for _ in range(R.N)] for q in E.q]
    ct = E.encrypt(s, a, m, e)
    keys = {}
    for gamma in range(0, alpha + 1):
        for h, _ in R.tower_steps(gamma):
            if h not in keys:
                ka = [[[rng.randrange(q) for _ in range(R.N)] for q in E.q] for _ in E.q]
                keys[h] = (ka, E.ksk(s, h, ka, [[0] * R.N for _ in E.q]))
        c = [0]
        out = E.hom_trace(ct, gamma, keys, c)
        assert c[0] == R.tower_ks_count(gamma)
        me = [x + y for x, y in zip(m, e)]
        want = R.partial_trace(me, gamma) if gamma >= 1 else R.trace(me)
        assert E.centered(E.decrypt(s, out)) == want, gamma
