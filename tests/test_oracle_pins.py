"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test names the independent fact it checks: a library routine (sympy,
numpy object-dtype polynomial products, Python big integers), a closed form
from the paper, a printed value (tests/golden/), or an exact algebraic
identity.  A dropped term, a wrong sign or index, or a transposed operand in
any oracle function makes at least one of them fail.
"""
import math
import os

import numpy as np
import pytest
import sympy

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _poly_eval(coeffs, x, q):
    """Horner evaluation with Python ints."""
    acc = 0
    for c in reversed([int(v) for v in coeffs]):
        acc = (acc * x + c) % q
    return acc


def _negacyclic_numpy(a, b, q):
    """Product with numpy's polymul on Python-int objects, folded by X^N = -1."""
    n = len(a)
    full = np.polymul(np.array([int(v) for v in a[::-1]], dtype=object),
                      np.array([int(v) for v in b[::-1]], dtype=object))[::-1]
    out = [0] * n
    for k, c in enumerate(full):
        if k < n:
            out[k] += int(c)
        else:
            out[k - n] -= int(c)
    return [v % q for v in out]


# ---------------------------------------------------------------- primes ----

@pytest.mark.parametrize("log_n,L,bits,K", [(12, 2, 30, 1), (14, 3, 50, 1), (15, 4, 50, 2), (16, 5, 50, 2)])
def test_primes_are_the_top_ntt_primes(oracle, log_n, L, bits, K):
    """sympy.isprime: every modulus is prime, 1 mod 2N, below 2^bits, and no
    such prime is skipped between 2^bits and the smallest one chosen."""
    prm = oracle.make_params(log_n, L, bits, K, bits)
    two_n = 2 * (1 << log_n)
    mods = prm.p + prm.q                      # generation order: special first
    assert len(set(mods)) == L + K
    for m in mods:
        assert sympy.isprime(m) and m % two_n == 1 and m < (1 << bits)
    k = ((1 << bits) - 2) // two_n
    expect = []
    while len(expect) < L + K:
        c = k * two_n + 1
        if sympy.isprime(c):
            expect.append(c)
        k -= 1
    assert mods == expect


def test_primitive_root(oracle):
    """psi^N = -1 and psi^(2N) = 1 (order exactly 2N)."""
    prm = oracle.make_params(10, 2, 50, 1, 50)
    for q in prm.mods:
        psi = oracle.lib().or_primitive_root_2n(q, 2 * prm.n)
        assert pow(psi, prm.n, q) == q - 1 and pow(psi, 2 * prm.n, q) == 1


# ------------------------------------------------------------- samplers -----

def test_splitmix64_reference_values(oracle):
    """Published SplitMix64 outputs (tests/golden/splitmix64.txt)."""
    for row in _read_golden("splitmix64.txt"):
        seed, vals = int(row[0]), [int(v) for v in row[1:]]
        got = [int(v) for v in oracle.splitmix64(seed, len(vals))]
        assert got == vals


def test_secret_and_noise_statistics(oracle):
    """Ternary secret: each of {-1,0,1} with frequency 1/3; rounded Gaussian:
    mean 0, standard deviation sqrt(sigma^2 + 1/12) (rounding adds 1/12)."""
    prm = oracle.make_params(16, 1, 50, 1, 50)
    s = oracle.keygen(prm, 11)
    assert set(np.unique(s)) <= {-1, 0, 1}
    for v in (-1, 0, 1):
        assert abs(np.mean(s == v) - 1 / 3) < 0.01
    a, e = oracle.sample_encrypt(prm, 12, 4)
    e = e.ravel().astype(np.float64)
    assert abs(e.mean()) < 0.05
    assert abs(e.std() - math.sqrt(3.2 ** 2 + 1 / 12)) < 0.05
    q = prm.q[0]
    assert a.max() < q and abs(a.mean() / q - 0.5) < 0.01


def test_permutation_is_uniform_bijection(oracle):
    """Fisher-Yates: a bijection, deterministic per (seed, round), different
    across rounds, and all 24 permutations of 4 items about equally likely."""
    p = oracle.permutation(5, 2, 1000)
    assert sorted(p.tolist()) == list(range(1000))
    assert (oracle.permutation(5, 2, 1000) == p).all()
    assert not (oracle.permutation(5, 3, 1000) == p).all()
    inv = oracle.inverse_perm(p)
    assert (p[inv] == np.arange(1000)).all()
    counts = {}
    for seed in range(24000):
        key = tuple(oracle.permutation(seed, 1, 4).tolist())
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 24
    chi2 = sum((c - 1000) ** 2 / 1000 for c in counts.values())
    assert chi2 < 60          # 23 dof; p ~ 5e-5


def test_quantize_rounds_half_away_from_zero(oracle):
    x = np.array([0.5, -0.5, 1.5, -1.5, 2.4999, -2.5001, 0.0])
    assert oracle.quantize(x, 1.0).tolist() == [1, -1, 2, -2, 2, -3, 0]
    assert oracle.quantize(np.array([0.75]), 2.0 ** 40).tolist() == [3 * 2 ** 38]


# ---------------------------------------------------------------- ring ------

@pytest.mark.parametrize("n,bits", [(1, 50), (2, 50), (8, 30), (64, 50)])
def test_polymul_matches_numpy_object_product(oracle, n, bits):
    """Schoolbook negacyclic product == numpy.polymul on Python ints folded
    by X^N = -1."""
    q = oracle.find_primes(2 * max(n, 2), bits, 1)[0]
    rng = np.random.default_rng(n)
    a = rng.integers(0, q, n, dtype=np.uint64)
    b = rng.integers(0, q, n, dtype=np.uint64)
    assert [int(v) for v in oracle.polymul(a, b, q)] == _negacyclic_numpy(a, b, q)


def test_polymul_evaluates_at_odd_powers_of_psi(oracle):
    """(a*b)(psi^k) = a(psi^k) b(psi^k) for odd k: the negacyclic ring is
    Z_q[X]/(X^N+1) whose roots are the odd powers of a primitive 2N-th root."""
    n = 256
    q = oracle.find_primes(2 * n, 50, 1)[0]
    psi = oracle.lib().or_primitive_root_2n(q, 2 * n)
    rng = np.random.default_rng(3)
    a = rng.integers(0, q, n, dtype=np.uint64)
    b = rng.integers(0, q, n, dtype=np.uint64)
    c = oracle.polymul(a, b, q)
    for k in (1, 3, 77, 2 * n - 1):
        x = pow(psi, k, q)
        assert _poly_eval(c, x, q) == _poly_eval(a, x, q) * _poly_eval(b, x, q) % q


def test_automorphism_by_evaluation_and_composition(oracle):
    """tau_d(a)(psi^k) = a(psi^(k d)); tau_a o tau_b = tau_(a b mod 2N)."""
    n = 64
    q = oracle.find_primes(2 * n, 50, 1)[0]
    psi = oracle.lib().or_primitive_root_2n(q, 2 * n)
    rng = np.random.default_rng(4)
    a = rng.integers(0, q, n, dtype=np.uint64)
    for d in (3, 5, 9, 2 * n - 1, n + 1):
        t = oracle.automorphism(a, d, q)
        for k in (1, 5, 31):
            assert _poly_eval(t, pow(psi, k, q), q) == _poly_eval(a, pow(psi, k * d, q), q)
    ab = oracle.automorphism(oracle.automorphism(a, 5, q), 9, q)
    assert (ab == oracle.automorphism(a, 45 % (2 * n), q)).all()


def test_monomial_mul(oracle):
    """X^s a == a * (the monomial X^s) by the numpy product, for s in [-2N, 2N]."""
    n = 16
    q = oracle.find_primes(2 * n, 50, 1)[0]
    rng = np.random.default_rng(5)
    a = rng.integers(0, q, n, dtype=np.uint64)
    for s in (0, 1, 7, n, n + 3, 2 * n - 1, -5):
        mono = [0] * n
        e = s % (2 * n)
        mono[e % n] = 1 if e < n else q - 1
        assert [int(v) for v in oracle.monomial_mul(a, s, q)] == _negacyclic_numpy(a, mono, q)


# ---------------------------------------------------------------- RLWE ------

def test_encrypt_decrypt_is_exact_up_to_sampled_noise(oracle):
    """Sec. 2.1: b = a s + m + e, so b - a s - m is exactly the sampled e."""
    prm = oracle.make_params(8, 3, 50, 1, 50)
    s = oracle.keygen(prm, 1)
    m = np.arange(2 * prm.n) * 7 - 900
    cts = oracle.encrypt(prm, s, m, 9, 2)
    _, e = oracle.sample_encrypt(prm, 9, 2)
    res = oracle.decrypt(prm, s, cts)
    for j in range(2):
        got = np.array(oracle.crt_centered(prm, res[j]), dtype=object)
        assert (got - m[j * prm.n:(j + 1) * prm.n] == e[j]).all()


def _crt(residues, moduli):
    M = math.prod(moduli)
    v = 0
    for r, m in zip(residues, moduli):
        mh = M // m
        v += int(r) * mh * pow(mh % m, -1, m)
    return v % M


@pytest.mark.parametrize("L,K", [(3, 1), (4, 2), (5, 2), (2, 1)])
def test_modup_is_fast_base_conversion(oracle, L, K):
    """Big-integer check of ModUp: the extended residues represent one integer
    X_j = x mod Q_j + u Q_j with 0 <= u < |D_j|, residue-exact on every modulus."""
    prm = oracle.make_params(4, L, 50, K, 50)
    rng = np.random.default_rng(L * 10 + K)
    x = np.stack([rng.integers(0, q, prm.n, dtype=np.uint64) for q in prm.q])
    for j in range(prm.dnum):
        D = list(prm.digit(j))
        Qj = math.prod(prm.q[i] for i in D)
        ext = oracle.modup(prm, j, x)
        for c in range(prm.n):
            xq = _crt([x[i, c] for i in D], [prm.q[i] for i in D])
            Xj = 0
            for i in D:
                qhat = Qj // prm.q[i]
                Xj += (int(x[i, c]) * pow(qhat % prm.q[i], -1, prm.q[i]) % prm.q[i]) * qhat
            assert (Xj - xq) % Qj == 0 and 0 <= (Xj - xq) // Qj < len(D)
            for m, qm in enumerate(prm.mods):
                assert int(ext[m, c]) == Xj % qm


@pytest.mark.parametrize("L,K", [(3, 1), (4, 2), (5, 2)])
def test_moddown_divides_by_p(oracle, L, K):
    """Big-integer check of ModDown: out = (X - conv_P(x_P)) / P mod q_i, where
    X is the CRT value over PQ and conv_P(x_P) = sum_k [x_pk Phat_k^-1]_pk Phat_k."""
    prm = oracle.make_params(4, L, 50, K, 50)
    rng = np.random.default_rng(L + K)
    x = np.stack([rng.integers(0, m, prm.n, dtype=np.uint64) for m in prm.mods])
    out = oracle.moddown(prm, x)
    P = prm.P
    for c in range(prm.n):
        X = _crt(x[:, c], prm.mods)
        conv = 0
        for k, pk in enumerate(prm.p):
            ph = P // pk
            conv += (int(x[L + k, c]) * pow(ph % pk, -1, pk) % pk) * ph
        assert (X - conv) % P == 0
        for i, qi in enumerate(prm.q):
            assert int(out[i, c]) == ((X - conv) // P) % qi


def test_rotation_key_decrypts_to_gadget_times_automorphed_secret(oracle):
    """Sec. 4.2: per digit j and modulus m, b_j - alpha_j s = e_j - [P g_j]_m s(X^d)
    with [g_j]_m = 1 on the digit's own data limbs, 0 elsewhere."""
    prm = oracle.make_params(6, 4, 50, 2, 50)
    s = oracle.keygen(prm, 3)
    d = 5
    key = oracle.rotkey(prm, s, 77, d)
    _, e = oracle.sample_rotkey(prm, 77, d)
    # s(X^d) by the evaluation definition checked above
    sd = [int(v) for v in oracle.automorphism(np.array(s) % prm.q[0], d, prm.q[0])]
    sd = [v - prm.q[0] if v > prm.q[0] // 2 else v for v in sd]
    for j in range(prm.dnum):
        for m, qm in enumerate(prm.mods):
            sa = oracle.polymul(key[j, 0, m], np.array(s) % qm, qm)
            diff = [(int(b) - int(a)) % qm for a, b in zip(sa, key[j, 1, m])]
            pg = 0
            if m < prm.L and m in prm.digit(j):
                pg = prm.P % qm
            want = [(int(e[j, k]) - pg * sd[k]) % qm for k in range(prm.n)]
            assert diff == want


@pytest.mark.parametrize("L,K", [(3, 1), (2, 1), (4, 2)])
def test_rotate_decrypts_to_automorphism_within_bound(oracle, L, K):
    """decrypt(rotate(ct, d)) = tau_d(m) + e_ks with
    |e_ks| <= N * sum_j |D_j| Q_j * 6 sigma / P + K (N + 1)  (fresh-noise
    term e' carries over as tau_d(e), |e| <= 6 sigma); trivial ciphertexts
    (a = 0) rotate exactly."""
    prm = oracle.make_params(7, L, 50, K, 50)
    s = oracle.keygen(prm, 5)
    keys = oracle.rotation_keys(prm, s, 8)
    m = (np.arange(prm.n) * 31337) % 100000 - 50000
    ct = oracle.encrypt(prm, s, m, 6, 1)[0]
    bound = prm.n * sum(len(prm.digit(j)) * math.prod(prm.q[i] for i in prm.digit(j))
                        for j in range(prm.dnum)) * 6 * prm.sigma / prm.P + K * (prm.n + 1) + 6 * prm.sigma
    for d in keys:
        got = np.array(oracle.crt_centered(prm, oracle.decrypt(prm, s, oracle.rotate(prm, keys, d, ct))[0]), dtype=object)
        want_res = np.stack([oracle.automorphism(np.asarray(m) % qi, d, qi) for qi in prm.q])
        want = np.array(oracle.crt_centered(prm, want_res), dtype=object)
        err = max(abs(int(v)) for v in got - want)
        assert err <= bound, (d, err, bound)
    triv = np.zeros((2, prm.L, prm.n), dtype=np.uint64)
    for i, qi in enumerate(prm.q):
        triv[1, i] = np.asarray(m) % qi
    for d in (3, 2 * prm.n // 2 + 1):
        r = oracle.rotate(prm, keys, d, triv)
        assert not r[0].any()
        for i, qi in enumerate(prm.q):
            assert (r[1, i] == oracle.automorphism(np.asarray(m) % qi, d, qi)).all()


# ------------------------------------------------------------- packing ------

def _trivial(prm, b_int):
    ct = np.zeros((2, prm.L, prm.n), dtype=np.uint64)
    for i, qi in enumerate(prm.q):
        ct[1, i] = np.array([int(v) % qi for v in b_int], dtype=np.uint64)
    return ct


@pytest.mark.parametrize("n", [1, 2, 4, 8, 32, 64])
def test_pack_of_trivial_ciphertexts_is_exact(oracle, n):
    """Sec. 2.4: packing n ciphertexts whose constant coefficients are m_l
    (all other coefficients garbage) gives exactly N * sum_l m_l X^(l N/n);
    the key-switch count is (n - 1) + log2(N/n)."""
    prm = oracle.make_params(7, 2, 50, 1, 50)
    s = oracle.keygen(prm, 1)
    keys = oracle.rotation_keys(prm, s, 2)
    rng = np.random.default_rng(n)
    bs = [rng.integers(-10 ** 6, 10 ** 6, prm.n) for _ in range(n)]
    c = oracle.Counter()
    out = oracle.pack(prm, keys, [_trivial(prm, b) for b in bs], c)
    assert not out[0].any()
    got = oracle.crt_centered(prm, out[1])
    want = [0] * prm.n
    for l in range(n):
        want[l * prm.n // n] = prm.n * int(bs[l][0])
    assert got == want
    assert c.ks == oracle.ks_count(prm, n) == (n - 1) + (prm.log_n - int(math.log2(n)))


def test_trace_of_monomials(oracle):
    """Sec. 2.3 closed form at t = 2: Tr(X^i) = N [i = 0] for the full trace
    (pack of a single ciphertext is the full trace)."""
    prm = oracle.make_params(6, 2, 50, 1, 50)
    s = oracle.keygen(prm, 1)
    keys = oracle.rotation_keys(prm, s, 2)
    for i in (0, 1, 5, prm.n - 1):
        b = [0] * prm.n
        b[i] = 1
        out = oracle.pack(prm, keys, [_trivial(prm, b)])
        got = oracle.crt_centered(prm, out[1])
        assert got == [prm.n if (k == 0 and i == 0) else 0 for k in range(prm.n)]


def test_encrypted_pack_decrypts_to_packed_messages(oracle):
    """Encrypted version of the pack pin: N m_l at l N/n, ~0 elsewhere, with
    noise far below the message scale."""
    prm = oracle.make_params(7, 3, 50, 1, 50)
    s = oracle.keygen(prm, 4)
    keys = oracle.rotation_keys(prm, s, 5)
    n = 8
    scale = 2 ** 40
    msgs = [(l - 3) * scale for l in range(n)]
    leaves = []
    for l in range(n):
        m = np.zeros(prm.n, dtype=np.int64)
        m[0] = msgs[l]
        m[1:] = np.arange(1, prm.n) * 1000      # garbage the trace must kill
        leaves.append(oracle.encrypt(prm, s, m, 100 + l, 1)[0])
    out = oracle.pack(prm, keys, leaves)
    got = oracle.crt_centered(prm, oracle.decrypt(prm, s, out)[0])
    for k in range(prm.n):
        want = prm.n * msgs[k // (prm.n // n)] if k % (prm.n // n) == 0 else 0
        assert abs(got[k] - want) < 2 ** 30


def test_ks_per_coefficient_matches_table1(oracle):
    """Table 1 of the paper, reproduced by the count formula of Sec. 2.4 to the
    printed two decimals."""
    for t, alpha, gamma, val in _read_golden("table1_ks_per_coefficient.txt"):
        got = oracle.ks_per_coefficient_general(int(t), int(alpha), int(gamma))
        assert abs(got - float(val)) <= 0.01, (t, alpha, gamma, got, val)


def test_ks_count_of_the_benchmark_layers(oracle):
    """One FC 64x64 layer at N = 2^12 packs 64 values with 63 merges and 6
    trace steps (69); a 16x32x32 conv at N = 2^14 gives 2 groups of 8192."""
    p1 = oracle.make_params(12, 2, 30, 1, 30)
    p2 = oracle.make_params(14, 3, 50, 1, 50)
    assert oracle.ks_count(p1, 64) == 69
    assert oracle.group_size(p2, 16384) == 8192
    assert oracle.ks_count(p2, 16384) == 16384


# -------------------------------------------------------- linear layer ------

def test_extracted_row_is_scaled_monomial_shift(oracle):
    """Sec. 4.4 (gamma = 0, t = 2): the row extracted for stream position
    p = jN + k is N^-1 X^-k ct_j; for a trivial ciphertext its constant
    coefficient is N^-1 m_k, and the full trace maps it back to m_k."""
    prm = oracle.make_params(6, 2, 50, 1, 50)
    s = oracle.keygen(prm, 1)
    keys = oracle.rotation_keys(prm, s, 2)
    rng = np.random.default_rng(9)
    m = rng.integers(-1000, 1000, 2 * prm.n)
    cts = np.stack([_trivial(prm, m[:prm.n]), _trivial(prm, m[prm.n:])])
    term = oracle.ConvTerm(0, 1, 1, 2 * prm.n, 2 * prm.n, 1, 1)
    W = np.eye(2 * prm.n).reshape(2 * prm.n, 1, 1, 2 * prm.n)
    lay = oracle.make_layer([term], [W], None, 1.0, 1.0)
    for i in (0, 3, prm.n - 1, prm.n, prm.n + 5):
        leaf = oracle.linear_output(prm, lay, cts, i)
        for li, qi in enumerate(prm.q):
            assert int(leaf[1, li, 0]) == int(m[i]) * pow(prm.n, -1, qi) % qi
        packed = oracle.pack(prm, keys, [leaf])
        assert oracle.crt_centered(prm, packed[1])[0] == int(m[i])


def _layer_case(oracle, prm, seed, H=4, W=4, C=3, Co=5, k=3, stride=1, pad=1, shortcut=False, bias=False,
                wscale=1.0, integer=True):
    rng = np.random.default_rng(seed)
    terms = [oracle.ConvTerm(0, H, W, C, Co, k, k, stride, pad)]
    if integer:
        ws = [rng.integers(-3, 4, (Co, k, k, C)).astype(np.float64)]
    else:
        ws = [rng.uniform(-1, 1, (Co, k, k, C))]
    if shortcut:
        t0 = terms[0]
        terms.append(oracle.ConvTerm(H * W * C, H, W, C, Co, 1, 1, stride, 0))
        ws.append(rng.integers(-2, 3, (Co, 1, 1, C)).astype(np.float64) if integer
                  else rng.uniform(-1, 1, (Co, 1, 1, C)))
        assert terms[1].H_out == t0.H_out
    b = rng.integers(-5, 6, Co).astype(np.float64) if bias else None
    return terms, ws, b


@pytest.mark.parametrize("case", ["conv", "strided+shortcut+bias", "fc"])
def test_layer_on_trivial_ciphertexts_equals_integer_matvec(oracle, case):
    """Noise-free check of the whole round (extract, unshuffle, linear,
    shuffle, pack, bias): the client reads exactly (A x + b)[sigma_out]
    where A is the layer's Toeplitz matrix built from the conv definition."""
    prm = oracle.make_params(8, 2, 50, 1, 50)
    s = oracle.keygen(prm, 1)
    keys = oracle.rotation_keys(prm, s, 2)
    if case == "conv":
        terms, ws, b = _layer_case(oracle, prm, 1, H=6, W=6, C=4, Co=4)
    elif case == "strided+shortcut+bias":
        terms, ws, b = _layer_case(oracle, prm, 2, H=6, W=6, C=3, Co=4, stride=2, shortcut=True, bias=True)
    else:
        terms = [oracle.ConvTerm(0, 1, 1, 150, 37, 1, 1)]
        ws = [np.random.default_rng(3).integers(-4, 5, (37, 1, 1, 150)).astype(np.float64)]
        b = None
    lay = oracle.make_layer(terms, ws, b, 1.0, 1.0)
    rng = np.random.default_rng(11)
    x = rng.integers(-50, 50, lay.E_in)
    sp = oracle.permutation(7, 1, lay.E_in)
    so = oracle.permutation(7, 2, lay.E_out)
    stream = x[sp]                                   # position k holds x[sigma_prev(k)]
    k_in = -(-lay.E_in // prm.n)
    padded = np.zeros(k_in * prm.n, dtype=np.int64)
    padded[:stream.size] = stream
    cts = np.stack([_trivial(prm, padded[j * prm.n:(j + 1) * prm.n]) for j in range(k_in)])
    out = oracle.eval_linear_layer(prm, lay, keys, cts, sp, so)
    vals = []
    n = oracle.group_size(prm, lay.E_out)
    for g in range(out.shape[0]):
        assert not out[g, 0].any()
        cent = oracle.crt_centered(prm, out[g, 1])
        cnt = min(n, lay.E_out - g * n)
        vals.extend(cent[l * (prm.n // n)] for l in range(cnt))
    A = oracle.dense_matrix(lay)
    y = A.dot(np.array([int(v) for v in x], dtype=object))
    if b is not None:
        y = y + np.array([int(b[o % lay.C_out]) for o in range(lay.E_out)], dtype=object)
    assert vals == [int(v) for v in y[so]]


def test_encrypted_layer_integer_mode_is_exact(oracle):
    """Sec. 6.1 correctness check: decrypting and rounding gives exactly the
    quantised cleartext result A xq, in the shuffled order."""
    prm = oracle.make_params(8, 3, 50, 1, 50)
    s = oracle.keygen(prm, 21)
    keys = oracle.rotation_keys(prm, s, 22)
    terms, ws, _ = _layer_case(oracle, prm, 5, H=5, W=5, C=4, Co=6)
    lay = oracle.make_layer(terms, ws, None, 1.0, 1.0)
    rng = np.random.default_rng(23)
    x = rng.integers(0, 16, lay.E_in)
    delta = 2 ** 30
    sp = oracle.permutation(24, 3, lay.E_in)
    so = oracle.permutation(24, 4, lay.E_out)
    cts = oracle.encrypt(prm, s, x[sp] * delta, 25, -(-lay.E_in // prm.n))
    out = oracle.eval_linear_layer(prm, lay, keys, cts, sp, so)
    res = oracle.decrypt(prm, s, out)
    n = oracle.group_size(prm, lay.E_out)
    got = []
    for g in range(res.shape[0]):
        cent = oracle.crt_centered(prm, res[g])
        cnt = min(n, lay.E_out - g * n)
        got.extend(round(cent[l * (prm.n // n)] / delta) for l in range(cnt))
    y = oracle.dense_matrix(lay).dot(np.array([int(v) for v in x], dtype=object))
    assert got == [int(v) for v in y[so]]


def test_encrypted_layer_float_mode_error(oracle):
    """Fixed-point mode: |decoded - W x| <= 1e-3 against float64 for U(-1,1)
    inputs and weights at scale 2^25 (inputs) x 2^25 (weights)."""
    prm = oracle.make_params(9, 2, 30, 1, 30)
    s = oracle.keygen(prm, 31)
    keys = oracle.rotation_keys(prm, s, 32)
    rng = np.random.default_rng(33)
    W = rng.uniform(-1, 1, (40, 1, 1, 40))
    x = rng.uniform(-1, 1, 40)
    lay = oracle.make_layer([oracle.ConvTerm(0, 1, 1, 40, 40, 1, 1)], [W], None, 2.0 ** 25, 2.0 ** 50)
    sp = oracle.permutation(34, 5, 40)
    so = oracle.permutation(34, 6, 40)
    cts = oracle.encrypt(prm, s, oracle.quantize(x[sp], 2.0 ** 25), 35, 1)
    out = oracle.eval_linear_layer(prm, lay, keys, cts, sp, so)
    got = oracle.read_outputs(prm, lay, oracle.decrypt(prm, s, out), 2.0 ** 50)
    ref = (W[:, 0, 0, :] @ x)[so]
    assert np.abs(got - ref).max() <= 1e-3


# ------------------------------------------------------ conv geometry ------
# The layer's geometry (receptive field, padding, stride, the channels-last
# flatten order (h W + w) C + c of Sec. 4.3, segment offsets of a second input)
# is checked against a convolution written out here from its definition:
# reshape the segment to an H x W x C_in image, zero-pad it, and for every
# kernel offset (dh, dw) add W[:, dh, dw, :] times the strided window of the
# padded image.  Nothing below calls the oracle's tap walk.

def _conv_direct(x, term, w):
    """y[ho, wo, co] = sum_{dh, dw, c} w[co, dh, dw, c] xpad[ho s + dh, wo s + dw, c],
    flattened channels last; x and w hold Python ints (object arrays)."""
    H, W, C, s, p = term.H, term.W, term.C_in, term.stride, term.pad
    img = np.asarray(x[term.in_offset:term.in_offset + H * W * C], dtype=object).reshape(H, W, C)
    xpad = np.zeros((H + 2 * p, W + 2 * p, C), dtype=object)
    xpad[p:p + H, p:p + W, :] = img
    Ho = (H + 2 * p - term.kh) // s + 1
    Wo = (W + 2 * p - term.kw) // s + 1
    y = np.zeros((Ho, Wo, term.C_out), dtype=object)
    for dh in range(term.kh):
        for dw in range(term.kw):
            win = xpad[dh:dh + s * (Ho - 1) + 1:s, dw:dw + s * (Wo - 1) + 1:s, :]   # Ho x Wo x C
            y += np.einsum("hwc,oc->hwo", win, np.asarray(w[:, dh, dw, :], dtype=object))
    return y.reshape(-1)


def _geometry_case(name):
    """(terms as tuples, weight shapes) of the geometry cases: a 3x3 stride-1
    pad-1 conv on a non-square input, a 3x3 stride-2 pad-1 conv on an odd
    non-square input, the 7x7 stride-2 pad-3 stem, and a block's second conv
    with a 1x1 stride-2 shortcut over a second input segment."""
    if name == "3x3s1p1":
        return [(0, 5, 6, 3, 4, 3, 1, 1)]
    if name == "3x3s2p1":
        return [(0, 7, 5, 2, 3, 3, 2, 1)]
    if name == "7x7s2p3":
        return [(0, 11, 9, 3, 4, 7, 2, 3)]
    if name == "3x3+1x1s2":
        # main conv over segment 0 (4x4x3 -> 4x4x5), shortcut 1x1 stride 2
        # over segment 1 (8x8x2 -> 4x4x5) starting at flat index 48
        return [(0, 4, 4, 3, 5, 3, 1, 1), (48, 8, 8, 2, 5, 1, 2, 0)]
    raise KeyError(name)


@pytest.mark.parametrize("name", ["3x3s1p1", "3x3s2p1", "7x7s2p3", "3x3+1x1s2"])
def test_layer_matrix_equals_direct_convolution(oracle, name):
    """The oracle's layer as a matrix (dense_matrix, built from its tap walk)
    times x equals the direct convolution of x, term by term, for every
    output; integer weights and inputs, compared exactly."""
    rng = np.random.default_rng(sum(map(ord, name)))
    terms, ws = [], []
    for (off, H, W, C, Co, k, s, p) in _geometry_case(name):
        terms.append(oracle.ConvTerm(off, H, W, C, Co, k, k, s, p))
        ws.append(rng.integers(-7, 8, (Co, k, k, C)).astype(np.float64))
    lay = oracle.make_layer(terms, ws, None, 1.0, 1.0)
    x = rng.integers(-100, 101, lay.E_in)
    xo = np.array([int(v) for v in x], dtype=object)
    want = sum(_conv_direct(xo, t, w.astype(np.int64)) for t, w in zip(terms, ws))
    got = oracle.dense_matrix(lay).dot(xo)
    assert list(got) == list(want)


def test_layer_round_over_several_ciphertexts_equals_direct_convolution(oracle):
    """A whole round on trivial ciphertexts whose input spans k_in = 3
    ciphertexts (positions j N + k after the unshuffle), with a strided 1x1
    shortcut over a second segment, bias, input unshuffle and output shuffle:
    the packed values read by the client equal the direct convolution plus
    bias, in shuffled order."""
    prm = oracle.make_params(6, 2, 50, 1, 50)             # N = 64
    s = oracle.keygen(prm, 41)
    keys = oracle.rotation_keys(prm, s, 42)
    rng = np.random.default_rng(43)
    terms = [oracle.ConvTerm(0, 5, 4, 4, 3, 3, 3, 2, 1),   # 5x4x4 -> 3x2x3
             oracle.ConvTerm(80, 6, 3, 5, 3, 1, 1, 2, 0)]  # 6x3x5 -> 3x2x3, second segment
    ws = [rng.integers(-5, 6, (3, 3, 3, 4)).astype(np.float64),
          rng.integers(-5, 6, (3, 1, 1, 5)).astype(np.float64)]
    b = rng.integers(-9, 10, 3).astype(np.float64)
    lay = oracle.make_layer(terms, ws, b, 1.0, 1.0)
    assert lay.E_in == 170 and -(-lay.E_in // prm.n) == 3
    x = rng.integers(-60, 61, lay.E_in)
    sp = oracle.permutation(44, 1, lay.E_in)
    so = oracle.permutation(44, 2, lay.E_out)
    stream = np.zeros(3 * prm.n, dtype=np.int64)
    stream[:lay.E_in] = x[sp]                               # position k holds x[sigma_prev(k)]
    cts = np.stack([_trivial(prm, stream[j * prm.n:(j + 1) * prm.n]) for j in range(3)])
    out = oracle.eval_linear_layer(prm, lay, keys, cts, sp, so)
    n = oracle.group_size(prm, lay.E_out)
    vals = []
    for g in range(out.shape[0]):
        cent = oracle.crt_centered(prm, out[g, 1])
        vals.extend(cent[l * (prm.n // n)] for l in range(min(n, lay.E_out - g * n)))
    xo = np.array([int(v) for v in x], dtype=object)
    y = sum(_conv_direct(xo, t, w.astype(np.int64)) for t, w in zip(terms, ws))
    y = y + np.array([int(b[o % 3]) for o in range(lay.E_out)], dtype=object)
    assert vals == [int(v) for v in y[so]]


# ---------------------------------------------------------------- noise ------
# The paper reports that the noise fast packing puts on each packed output is
# Gaussian-shaped and far inside the decryption bound (Sec. 5, Remark on DP
# amplification; appendix "FHE Noise").  These pins derive the first two
# moments of that noise from the key-switching definition and compare them
# with the oracle over many seeds.
#
# One key switch of tau_d(c) adds, per coefficient,
#     e_ks = sum_j ct_j * e_j / P  -  IH_B  +  IH_A * s          (real, then floored)
# where ct_j is the ModUp of digit j (an integer in [0, |D_j| Q_j), sum of
# |D_j| uniform terms), e_j the key noise (rounded Gaussian, variance
# sigma^2 + 1/12), and IH_A, IH_B the ModDown remainders x_P / P plus the
# fast-base-conversion overflow: a sum of K uniforms on [0, 1) (Irwin-Hall).
# With s uniform ternary (E s^2 = 2/3):
#     mean  -K/2
#     var   N (sigma^2 + 1/12) sum_j E[ct_j^2] / P^2 + N (K/12 + K^2/4) (2/3) + K/12
#     E[ct_j^2] = |D_j| Q_j^2 / 3 + |D_j| (|D_j| - 1) Q_j^2 / 4.
# Across two key switches under the same secret with independent masks only
# the IH_A * s terms correlate: E IH_A = K/2, and for positions p, p'
#     cov = (K^2 / 4)(2/3) sum_i F_p(i) F_p'(i) = (K^2 / 6)(N - 2 |p - p'|),
# F_p(i) = +1 for i <= p, -1 otherwise (the negacyclic signs of 1 * s).
#
# Packing (t = 2, gamma = 0): at a packed position the tree gives
# e <- e_ks + 2 e_child (tau_{m+1} fixes even lattice points and negates odd
# ones, which the X^s shift of the odd half cancels) and every trace step
# gives e <- 2 e + e_ks (tau_{2^k+1} fixes the whole lattice).  So the
# noise at position l N / n is sum_k w_k e_ks,k[p_k] over the log2 n tree
# merges on leaf l's path (weights 2^T, 2^(T+1), ..., positions moving down
# by N/m where leaf l's bit at that level is odd) and the T = log2(N/n) trace
# steps (weights 2^(T-1), ..., 1, all at l N / n), each key switch under its
# own key.

def _ks_noise_moments(prm):
    """(mean, variance) of one key switch's noise per coefficient."""
    N, K = prm.n, prm.K
    sig2 = prm.sigma ** 2 + 1.0 / 12
    ct2 = 0.0
    for j in range(prm.dnum):
        D = list(prm.digit(j))
        Qj = math.prod(prm.q[i] for i in D)
        ct2 += (len(D) * Qj ** 2 / 3 + len(D) * (len(D) - 1) * Qj ** 2 / 4) / prm.P ** 2
    return -K / 2, N * sig2 * ct2 + N * (K / 12 + K * K / 4) * (2.0 / 3) + K / 12


def _packed_noise_moments(prm, n, l):
    """(mean, variance) of the noise at packed position l N / n."""
    N, K = prm.n, prm.K
    T = prm.log_n - int(math.log2(n))
    p = l * N // n
    path = [(2 ** (T - t), p) for t in range(1, T + 1)]          # trace steps
    m, lm, w = n, l, 2 ** T
    while m >= 2:                                                 # tree merges, root first
        path.append((w, p))
        if lm % 2:
            p -= N // m
        lm, m, w = lm // 2, m // 2, 2 * w
    mu, v = _ks_noise_moments(prm)
    var = v * sum(wk * wk for wk, _ in path)
    for a, (wa, pa) in enumerate(path):
        for b, (wb, pb) in enumerate(path):
            if a != b:
                var += wa * wb * (K * K / 6.0) * (N - 2 * abs(pa - pb))
    return mu * sum(wk for wk, _ in path), var


def _noise_free(oracle, prm, s, msg, seed):
    """A ciphertext (a, a s + m) with uniform mask and no noise."""
    import dataclasses
    return oracle.encrypt(dataclasses.replace(prm, sigma=0.0), s, msg, seed, 1)[0]


def _seed_stats(samples):
    """Pooled mean and second central moment over seeds, with standard errors
    from the spread of the per-seed values (seeds are independent)."""
    x = np.array(samples, dtype=np.float64)           # [seeds][values per seed]
    m1 = x.mean(axis=1)
    mean = m1.mean()
    m2 = (x ** 2).mean(axis=1)
    var = m2.mean() - mean ** 2
    return mean, m1.std() / np.sqrt(len(x)), var, m2.std() / np.sqrt(len(x))


@pytest.mark.parametrize("L,qbits,K,pbits", [(3, 50, 1, 50), (3, 50, 2, 50), (2, 30, 1, 60), (2, 30, 2, 60)])
def test_keyswitch_noise_moments(oracle, L, qbits, K, pbits):
    """Mean and variance of the noise one key switch adds (rotation of a
    noise-free ciphertext by tau_3) match the analytic model above, for
    one-limb and two-limb digits, with P about Q_j (key noise dominates) and
    with P >> Q (ModDown remainders dominate); 600 seeds of key and mask."""
    prm = oracle.make_params(8, L, qbits, K, pbits)
    d = 3
    samples = []
    for sd in range(600):
        s = oracle.keygen(prm, 1000 + sd)
        keys = oracle.rotation_keys(prm, s, 2000 + sd, [d])
        m = np.random.default_rng(sd).integers(-1000, 1001, prm.n)
        r = oracle.rotate(prm, keys, d, _noise_free(oracle, prm, s, m, 3000 + sd))
        got = oracle.crt_centered(prm, oracle.decrypt(prm, s, r)[0])
        tm = [0] * prm.n                               # tau_d(m) by its definition
        for i in range(prm.n):
            e = i * d % (2 * prm.n)
            if e < prm.n:
                tm[e] += int(m[i])
            else:
                tm[e - prm.n] -= int(m[i])
        samples.append([g - t for g, t in zip(got, tm)])
    mean, se_mean, var, se_var = _seed_stats(samples)
    mu, v = _ks_noise_moments(prm)
    assert abs(mean - mu) <= 4 * se_mean + 0.05, (mean, mu, se_mean)
    assert abs(var - v) <= 4 * se_var, (var, v, se_var)
    assert abs(var / v - 1) <= 0.12


@pytest.mark.parametrize("L,qbits,K,pbits", [(3, 50, 2, 50), (2, 30, 1, 60)])
def test_packed_noise_moments_shape_and_bound(oracle, L, qbits, K, pbits):
    """Noise of fast packing on noise-free leaves (N = 256, n = 8, 300 seeds):
    at every packed position its mean and variance match the path model
    above; pooled over positions it is Gaussian-shaped (skewness and excess
    kurtosis near 0); and every coefficient of every output lies far inside
    the decryption bound Q/2."""
    prm = oracle.make_params(8, L, qbits, K, pbits)
    n = 8
    per_pos = [[] for _ in range(n)]
    worst = 0
    for sd in range(300):
        s = oracle.keygen(prm, 5000 + sd)
        keys = oracle.rotation_keys(prm, s, 6000 + sd)
        leaves = [_noise_free(oracle, prm, s, np.zeros(1, dtype=np.int64), 7000 + 100 * sd + l) for l in range(n)]
        dec = oracle.crt_centered(prm, oracle.decrypt(prm, s, oracle.pack(prm, keys, leaves))[0])
        worst = max(worst, max(abs(v) for v in dec))
        for l in range(n):
            per_pos[l].append([dec[l * prm.n // n]])
    z = []
    for l in range(n):
        mean, se_mean, var, se_var = _seed_stats(per_pos[l])
        mu, v = _packed_noise_moments(prm, n, l)
        assert abs(mean - mu) <= 4 * se_mean, (l, mean, mu, se_mean)
        assert abs(var - v) <= 4 * se_var, (l, var, v, se_var)
        z.extend((np.array(per_pos[l])[:, 0] - mu) / math.sqrt(v))
    z = np.array(z)
    skew = np.mean(z ** 3) / np.mean(z ** 2) ** 1.5
    exkurt = np.mean(z ** 4) / np.mean(z ** 2) ** 2 - 3
    assert abs(skew) < 0.2 and abs(exkurt) < 0.5, (skew, exkurt)
    std_max = max(math.sqrt(_packed_noise_moments(prm, n, l)[1]) for l in range(n))
    assert worst < 8 * std_max < prm.Q / 2 ** 20


# ------------------------------------------------ partial trace, gamma = 2 ---
# At t = 2 the tower is K_0 = K_1 = Q, K_2 = Q(i), ..., K_alpha = K.  The
# partial trace over K_2 / K_0 sums the automorphisms {1, 3} (Lemma 1, j in
# {0, 1}, k = 1), and the rest of the full trace is the sum over
# Gal(K / K_2) = {d = 1 mod 4}, generated by the tau_{2^k+1} with k >= 2.

def _tau_int(v, d, n):
    """tau_d on an integer coefficient vector, from its definition
    X^i -> X^(i d mod 2N) with X^N = -1."""
    out = [0] * n
    for i, c in enumerate(v):
        e = i * d % (2 * n)
        if e < n:
            out[e] += int(c)
        else:
            out[e - n] -= int(c)
    return out


def test_client_power_is_evaluation_at_cubes(oracle):
    """The client's power m(X^3) (Sec. 4.3, gamma = 2, t = 2) evaluates at every
    odd power of psi to m at the cube of that point."""
    prm = oracle.make_params(5, 1, 50, 1, 50)
    q = prm.q[0]
    psi = oracle.lib().or_primitive_root_2n(q, 2 * prm.n)
    m = np.random.default_rng(1).integers(-1000, 1001, prm.n)
    m3 = oracle.client_power(prm, m)
    for e in range(1, 2 * prm.n, 2):
        x = pow(psi, e, q)
        assert _poly_eval([int(v) % q for v in m3], x, q) == _poly_eval([int(v) % q for v in m], pow(x, 3, q), q)


def test_lemma1_gamma2_extraction(oracle):
    """Lemma 1 at t = 2, gamma = 2: the constant coefficient of
    X^-i m(X) + X^-3i m(X^3) is 2 m_i, so the extracted row (its scaling by
    (N/2)^-1) has constant coefficient 4 m_i / N; the remaining trace over
    K / K_2 (packing one value, log2 N - 1 key switches) maps the row to
    exactly 2 m_i = [K_2 : K_0] m_i with every other coefficient zero."""
    prm = oracle.make_params(6, 2, 50, 1, 50)
    s = oracle.keygen(prm, 1)
    keys = oracle.rotation_keys(prm, s, 2)
    m = np.random.default_rng(3).integers(-10 ** 6, 10 ** 6, prm.n)
    ct, ct3 = _trivial(prm, m), _trivial(prm, oracle.client_power(prm, m))
    for i in (0, 1, 7, prm.n - 1):
        row = oracle.extract(prm, ct, i, 2, ct3)
        for li, qi in enumerate(prm.q):
            assert int(row[1, li, 0]) == 4 * int(m[i]) * pow(prm.n, -1, qi) % qi
        c = oracle.Counter()
        out = oracle.pack(prm, keys, [row], c, gamma=2)
        assert oracle.crt_centered(prm, out[1]) == [2 * int(m[i]) if k == 0 else 0 for k in range(prm.n)]
        assert c.ks == prm.log_n - 1


@pytest.mark.parametrize("n", [1, 2, 4, 8, 32])
def test_pack_gamma2_of_partial_traces(oracle, n):
    """Packing leaves that hold y_l + tau_3(y_l) at gamma = 2 gives exactly the
    gamma = 0 packing of the y_l, N sum_l y_l[0] X^(l N / n), with n/2 fewer
    key switches (one fewer when n = 1)."""
    prm = oracle.make_params(7, 2, 50, 1, 50)
    s = oracle.keygen(prm, 1)
    keys = oracle.rotation_keys(prm, s, 2)
    rng = np.random.default_rng(100 + n)
    ys = [rng.integers(-10 ** 5, 10 ** 5, prm.n) for _ in range(n)]
    y2 = [[int(a) + b for a, b in zip(y, _tau_int(y, 3, prm.n))] for y in ys]
    c0, c2 = oracle.Counter(), oracle.Counter()
    out0 = oracle.pack(prm, keys, [_trivial(prm, y) for y in ys], c0)
    out2 = oracle.pack(prm, keys, [_trivial(prm, y) for y in y2], c2, gamma=2)
    assert (out0 == out2).all()
    want = [0] * prm.n
    for l in range(n):
        want[l * prm.n // n] = prm.n * int(ys[l][0])
    assert oracle.crt_centered(prm, out2[1]) == want
    assert c0.ks - c2.ks == (n // 2 if n >= 2 else 1)
    assert c2.ks == oracle.ks_count(prm, n, gamma=2)


def test_encrypted_layer_gamma2_integer_mode_is_exact(oracle):
    """A whole encrypted round at gamma = 2 (the client also sends RLWE(m(X^3))
    per input ciphertext): decrypting and halving (the [K_2 : K_0] factor)
    gives exactly the quantised A x + b in shuffled order, with the gamma = 2
    key-switch count."""
    prm = oracle.make_params(8, 3, 50, 1, 50)
    s = oracle.keygen(prm, 21)
    keys = oracle.rotation_keys(prm, s, 22)
    terms, ws, b = _layer_case(oracle, prm, 5, H=5, W=5, C=4, Co=6, bias=True)
    delta = 2 ** 30
    lay = oracle.make_layer(terms, ws, b, 1.0, float(delta))
    rng = np.random.default_rng(23)
    x = rng.integers(0, 16, lay.E_in)
    sp = oracle.permutation(24, 3, lay.E_in)
    so = oracle.permutation(24, 4, lay.E_out)
    k_in = -(-lay.E_in // prm.n)
    stream = np.zeros(k_in * prm.n, dtype=np.int64)
    stream[:lay.E_in] = x[sp] * delta
    cts = oracle.encrypt(prm, s, stream, 25, k_in)
    powers = np.stack([oracle.encrypt(prm, s, oracle.client_power(prm, stream[j * prm.n:(j + 1) * prm.n]),
                                      26 + j, 1)[0] for j in range(k_in)])
    c = oracle.Counter()
    out = oracle.eval_linear_layer(prm, lay, keys, cts, sp, so, c, powers=powers)
    assert c.ks == oracle.ks_count(prm, lay.E_out, gamma=2) < oracle.ks_count(prm, lay.E_out)
    res = oracle.decrypt(prm, s, out)
    n = oracle.group_size(prm, lay.E_out)
    got = []
    for g in range(res.shape[0]):
        cent = oracle.crt_centered(prm, res[g])
        got.extend(round(cent[l * (prm.n // n)] / (2 * delta)) for l in range(min(n, lay.E_out - g * n)))
    y = oracle.dense_matrix(lay).dot(np.array([int(v) for v in x], dtype=object))
    y = y + np.array([int(b[o % lay.C_out]) for o in range(lay.E_out)], dtype=object)
    assert got == [int(v) for v in y[so]]
