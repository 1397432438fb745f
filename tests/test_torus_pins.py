"""Pins of the torus RLWE oracle (oracle/primepower.py, TorusRlwe: the
paper's scheme over T_q, q = 2^53, Sec. 2.1-2.3 and Sec. 4.2, with the
gadget parameters of Table 2) to facts that do not come from it: the exact
product of Ring.mul, a brute-force nearest-digit search for the gadget
decomposition, exact rational bounds, a gadget that is exact when D^l
divides q (the key switch is then the automorphism itself), the trace by
definition, the predicted variance of the key-switching noise, and the
decryption boundary 1 / (2p) of Sec. 2.1 at Table 2's parameters."""
import itertools
import math
import random
from fractions import Fraction

import pytest

from oracle import primepower as pp

Q = 2 ** 53

# Table 2: (precision b, gamma column) -> t, alpha, D, l, noise Delta = 2^-x
TABLE2 = {
    (8, 0): (3, 7, 512, 3, 36), (8, 1): (3, 7, 512, 3, 36),
    (12, 0): (7, 4, 2 ** 12, 3, 51), (12, 1): (7, 4, 2 ** 16, 2, 51),
    (16, 0): (5, 5, 310, 5, 51), (16, 1): (5, 5, 310, 4, 51),
}


def _torus_dist(x, y):
    """Distance on R / Z between two Fractions."""
    d = (x - y) % 1
    return min(d, 1 - d)


def _ternary(rng, n):
    return [rng.choice((-1, 0, 1)) for _ in range(n)]


@pytest.mark.parametrize("t,alpha", [(3, 3), (5, 2), (7, 2)])
def test_product_is_the_exact_ring_product_mod_q(t, alpha):
    """The uint64 schoolbook product equals Ring.mul (exact Python integers)
    reduced mod 2^53, for torus-by-small and for large signed operands."""
    R = pp.Ring(t, alpha)
    T = pp.TorusRlwe(R, 512, 3)
    rng = random.Random(7 * t + alpha)
    for lo, hi in ((0, Q - 1), (-2 ** 62, 2 ** 62)):
        a = [rng.randint(lo, hi) for _ in range(R.N)]
        b = [rng.randint(-300, 300) for _ in range(R.N)]
        c = [rng.randint(-2 ** 60, 2 ** 60) for _ in range(R.N)]
        assert T.mul(a, b) == R.mod(R.mul(a, b), Q)
        assert T.mul(a, c) == R.mod(R.mul(a, c), Q)


@pytest.mark.parametrize("D,l", [(3, 2), (4, 3), (5, 3), (8, 2), (7, 3)])
def test_decomposition_is_the_nearest_digit_tuple(D, l):
    """For small gadgets every digit tuple in [-floor(D/2), D - floor(D/2))^l is
    tried: the decomposition is the one whose sum_i d_i / D^i is nearest to
    x / q on the torus (ties excluded)."""
    T = pp.TorusRlwe(pp.Ring(3, 2), D, l)
    rng = random.Random(D * 10 + l)
    half = D // 2
    xs = [rng.randrange(Q) for _ in range(60)] + [0, 1, Q - 1, Q // 2, Q // 3, (Q // D ** l) * 5]
    tuples = list(itertools.product(range(-half, D - half), repeat=l))
    for x in xs:
        target = Fraction(x, Q)
        dist = sorted((_torus_dist(target, sum(Fraction(d, D ** (i + 1)) for i, d in enumerate(tp))), tp)
                      for tp in tuples)
        if dist[0][0] == dist[1][0]:
            continue
        got = tuple(row[0] for row in T.decompose([x]))
        assert got == dist[0][1], (x, got, dist[0])


@pytest.mark.parametrize("D,l", [(512, 3), (2 ** 12, 3), (2 ** 16, 2), (310, 5), (310, 4), (3, 20)])
def test_decomposition_error_and_digit_range(D, l):
    """Table 2's gadgets: digits in range, and sum_i d_i / D^i within
    1 / (2 D^l) of x / q on the torus (exact rationals)."""
    T = pp.TorusRlwe(pp.Ring(3, 2), D, l)
    rng = random.Random(D + l)
    xs = [rng.randrange(Q) for _ in range(300)] + [0, 1, Q - 1, Q // 2, Q // 2 - 1, Q // 2 + 1]
    digits = T.decompose(xs)
    half = D // 2
    for k, x in enumerate(xs):
        ds = [digits[i][k] for i in range(l)]
        assert all(-half <= d < D - half for d in ds)
        approx = sum(Fraction(d, D ** (i + 1)) for i, d in enumerate(ds))
        assert _torus_dist(Fraction(x, Q), approx) <= Fraction(1, 2 * D ** l)


def test_power_of_two_gadget_digits_are_bit_fields():
    """With D = 2^k and D^l dividing q, x a multiple of q / D^l: the digits
    are the k-bit fields of x / (q / D^l), read as balanced digits."""
    k, l = 9, 3
    T = pp.TorusRlwe(pp.Ring(3, 2), 2 ** k, l)
    rng = random.Random(5)
    for _ in range(200):
        y = rng.randrange(2 ** (k * l))
        x = y << (53 - k * l)
        fields = [(y >> (k * (l - 1 - i))) & (2 ** k - 1) for i in range(l)]
        # balanced: a field >= 2^(k-1) becomes negative and carries into the next field up
        bal, carry = [0] * l, 0
        for i in range(l - 1, -1, -1):
            f = fields[i] + carry
            carry = 1 if f >= 2 ** (k - 1) else 0
            bal[i] = f - (2 ** k if carry else 0)
        assert [row[0] for row in T.decompose([x])] == bal


@pytest.mark.parametrize("D", [512, 310, 2 ** 12])
def test_gadget_message_rounding(D):
    """round(c q / D^i): within 1/2 of the rational value; exact for D = 2^9."""
    T = pp.TorusRlwe(pp.Ring(3, 2), D, 3)
    cs = list(range(-4, 5))
    for i in (1, 2, 3):
        g = T.gadget_message(cs, i)
        for c, v in zip(cs, g):
            exact = Fraction(c * Q, D ** i)
            rep = v if v < Q // 2 else v - Q
            assert abs(rep - exact) <= Fraction(1, 2)
            if D == 512:
                assert rep == c * 2 ** (53 - 9 * i)


def test_encode_decode_boundary():
    """pi_p of Sec. 2.1: decoding is correct exactly for noise in
    [-q/(2p), q/(2p)) (halves rounded up), p = 2^b for the b of Table 2."""
    T = pp.TorusRlwe(pp.Ring(3, 2), 512, 3)
    for b in (8, 12, 16):
        p = 2 ** b
        mu = [0, 1, p // 2, p - 1, 77]
        m = T.encode(mu, b)
        assert m == [v * (Q // p) for v in mu]
        lim = Q // (2 * p)
        for e, ok in ((0, True), (lim - 1, True), (-lim, True), (lim, False), (-lim - 1, False)):
            dec = T.decode([(x + e) % Q for x in m], b)
            assert (dec == mu) == ok, (b, e)


@pytest.mark.parametrize("t,alpha", [(3, 3), (5, 2)])
def test_encrypt_decrypt_phase_is_message_plus_noise(t, alpha):
    R = pp.Ring(t, alpha)
    T = pp.TorusRlwe(R, 512, 3)
    rng = random.Random(t)
    s = _ternary(rng, R.N)
    a = [rng.randrange(Q) for _ in range(R.N)]
    m = T.encode([rng.randrange(256) for _ in range(R.N)], 8)
    e = [rng.randint(-2 ** 17, 2 ** 17) for _ in range(R.N)]
    ct = T.encrypt(s, a, m, e)
    assert T.decrypt(s, ct) == [(x + y) % Q for x, y in zip(m, e)]
    # b - a s by the exact ring product, independently of TorusRlwe.mul
    assert ct[1] == [(x + y + z) % Q for x, y, z in zip(R.mul(a, s), m, e)]


@pytest.mark.parametrize("t,alpha,D,l", [(3, 3, 512, 3), (5, 2, 2 ** 12, 3), (7, 2, 2 ** 16, 2)])
def test_keyswitch_is_the_automorphism_when_the_gadget_is_exact(t, alpha, D, l):
    """D^l divides q and tau_h(a) is a multiple of q / D^l, noiseless keys:
    then sum_i d_i / D^i = tau_h(a) / q exactly, every key message is exact,
    and the key switch decrypts to tau_h of the phase, exactly."""
    R = pp.Ring(t, alpha)
    T = pp.TorusRlwe(R, D, l)
    step = Q // D ** l
    rng = random.Random(11 * t + l)
    s = _ternary(rng, R.N)
    a = [rng.randrange(D ** l) * step for _ in range(R.N)]
    m = [rng.randrange(Q) for _ in range(R.N)]
    e = [rng.randint(-50, 50) for _ in range(R.N)]
    ct = T.encrypt(s, a, m, e)
    phase = T.decrypt(s, ct)
    for h in R.units()[1:6]:
        ka = [[rng.randrange(Q) for _ in range(R.N)] for _ in range(l)]
        kb = T.ksk(s, h, ka, [[0] * R.N for _ in range(l)])
        out = T.keyswitch(ct, h, ka, kb)
        assert T.decrypt(s, out) == R.mod(R.automorphism(phase, h), Q)


@pytest.mark.parametrize("t,alpha", [(3, 3), (5, 2), (7, 2)])
def test_hom_trace_is_the_trace_when_the_gadget_is_exact(t, alpha):
    """With a and every ka a multiple of q / D^l (D = 512, l = 3) and
    noiseless keys, each intermediate mask stays a multiple of q / D^l, so the
    homomorphic tower trace decrypts exactly to the trace by definition (full
    trace at gamma = 0, Tr_{K / K_gamma} above) of the phase, with the tower's
    key-switch count."""
    R = pp.Ring(t, alpha)
    D, l = 512, 3
    T = pp.TorusRlwe(R, D, l)
    step = Q // D ** l
    rng = random.Random(3 * t + alpha)
    s = _ternary(rng, R.N)
    ct = T.encrypt(s, [rng.randrange(D ** l) * step for _ in range(R.N)], [rng.randrange(Q) for _ in range(R.N)],
                   [rng.randint(-9, 9) for _ in range(R.N)])
    phase = T.decrypt(s, ct)
    for gamma in range(0, alpha + 1):
        keys = {}
        for h, _ in R.tower_steps(gamma):
            ka = [[rng.randrange(D ** l) * step for _ in range(R.N)] for _ in range(l)]
            keys[h] = (ka, T.ksk(s, h, ka, [[0] * R.N for _ in range(l)]))
        cnt = [0]
        out = T.hom_trace(ct, gamma, keys, cnt)
        want = R.trace(phase) if gamma == 0 else R.partial_trace(phase, gamma)
        assert T.decrypt(s, out) == R.mod(want, Q)
        assert cnt[0] == R.tower_ks_count(gamma)


def _pair_counts(R):
    """#{(u, v): u, v < N, u + v = j (mod M)} for every j < M (brute force)."""
    cnt = [0] * R.M
    for u in range(R.N):
        for v in range(R.N):
            cnt[(u + v) % R.M] += 1
    return cnt


@pytest.mark.parametrize("t,alpha,D,l", [(3, 4, 2 ** 12, 4), (5, 3, 2 ** 8, 6)])
def test_keyswitch_noise_variance(t, alpha, D, l):
    """Key noise of standard deviation sigma dominates (the gadget's own
    rounding is below 2^5): the key-switch noise tau_h(phase) - phase' has
    per-coefficient variance l E[d^2] sigma^2 (#c_i + #c_(N + i mod m)) / N on
    average, #c_j the pairs (u, v) with u + v = j (mod M) (coefficient i of a
    product reduced mod Phi_M is c_i - c_(N + i mod m)), E[d^2] = (D^2 + 2) / 12
    for digits uniform on [-D/2, D/2).  Checked within 20 % over 4 seeds, and
    the noise has mean ~ 0."""
    R = pp.Ring(t, alpha)
    T = pp.TorusRlwe(R, D, l)
    sigma = 2.0 ** 16
    cnt = _pair_counts(R)
    terms = sum(cnt[i] + cnt[R.N + i % R.m] for i in range(R.N)) / R.N
    pred = l * (D * D + 2) / 12 * sigma ** 2 * terms
    rng = random.Random(101 + t)
    sq, tot, n = 0.0, 0.0, 0
    for seed in range(4):
        s = _ternary(rng, R.N)
        ct = T.encrypt(s, [rng.randrange(Q) for _ in range(R.N)], [0] * R.N, [0] * R.N)
        h = R.units()[1 + seed]
        ka = [[rng.randrange(Q) for _ in range(R.N)] for _ in range(l)]
        e = [[round(rng.gauss(0.0, sigma)) for _ in range(R.N)] for _ in range(l)]
        kb = T.ksk(s, h, ka, e)
        noise = T.centered([(x - y) % Q for x, y in zip(T.decrypt(s, T.keyswitch(ct, h, ka, kb)),
                                                         R.mod(R.automorphism(T.decrypt(s, ct), h), Q))])
        sq += sum(float(v) ** 2 for v in noise)
        tot += sum(float(v) for v in noise)
        n += len(noise)
    var = sq / n
    assert abs(var / pred - 1) < 0.2, (var, pred)
    assert abs(tot / n) < 4 * math.sqrt(pred / n)


@pytest.mark.parametrize("b,gamma", [(8, 0), (12, 0), (12, 1), (16, 0), (16, 1)])
def test_table2_trace_decrypts_within_the_boundary(b, gamma):
    """Table 2's rings, gadgets and noise: a message of b bits, encrypted with
    Gaussian noise of standard deviation Delta q, keys with the same noise; the
    homomorphic trace (full at gamma = 0, Tr_{K / K_1} in the gamma in [1, 2]
    column) decodes to the trace of the message mod p = 2^b, and its noise
    stays below q / (2p) (Sec. 2.1, the decryption condition).  The margin is
    about 2x at b = 16 with l = 4, where the gadget's rounding (q / (2 D^l) =
    2^18.9 per coefficient of tau_h(a)) dominates, and 2^6 or more elsewhere."""
    t, alpha, D, l, dx = TABLE2[(b, gamma)]
    R = pp.Ring(t, alpha)
    T = pp.TorusRlwe(R, D, l)
    sigma = Q * 2.0 ** -dx
    rng = random.Random(b * 10 + gamma)
    s = _ternary(rng, R.N)
    mu = [rng.randrange(2 ** b) for _ in range(R.N)]
    ct = T.encrypt(s, [rng.randrange(Q) for _ in range(R.N)], T.encode(mu, b),
                   [round(rng.gauss(0.0, sigma)) for _ in range(R.N)])
    keys = {}
    for h, _ in R.tower_steps(gamma):
        ka = [[rng.randrange(Q) for _ in range(R.N)] for _ in range(l)]
        e = [[round(rng.gauss(0.0, sigma)) for _ in range(R.N)] for _ in range(l)]
        keys[h] = (ka, T.ksk(s, h, ka, e))
    out = T.hom_trace(ct, gamma, keys)
    want = R.tower_trace(mu, gamma)
    phase = T.decrypt(s, out)
    noise = T.centered([(x - y) % Q for x, y in zip(phase, T.encode(want, b))])
    assert max(abs(v) for v in noise) < Q // (2 * 2 ** b)
    assert T.decode(phase, b) == [v % 2 ** b for v in want]
