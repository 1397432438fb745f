"""Plain CPU oracle for the paper's prime-power cyclotomic rings (Sec. 2.1,
2.3, 2.4; Table 2 lists M in {3^7, 7^4, 5^5}).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/`` may
import it; the product path never does.  Everything here is exact (Python
integers, and fractions where the dual basis needs them) and follows the
definitions literally:

* K = Q[X] / Phi_M(X), M = t^alpha with t prime, N = phi(M) = (t - 1) t^(alpha-1);
  Phi_M(X) = sum_{k < t} X^(k M / t), so X^N = -sum_{k < t-1} X^(k M / t).
* tau_d: P(X) -> P(X^d) mod Phi_M for gcd(d, M) = 1 (Sec. 2.2).
* Tr(P) = sum over gcd(d, M) = 1 of tau_d(P) (Sec. 2.3), and the partial
  traces Tr_{K / K_i} over Gal(K / K_i) = {d = 1 mod t^i}, K_i = Q(zeta_{t^i}).
* The tower evaluation of the full trace (Sec. 2.3): for i = alpha-1 down to
  1 the step Tr_{K_{i+1} / K_i} sums the t powers of tau_{1 + t^i} (t - 1
  automorphisms each), then Tr_{K_1 / K_0} over the cyclic group
  (Z / tZ)^* is taken one prime factor l of t - 1 at a time, each step
  summing l powers of one automorphism (l - 1 of them): in all
  (alpha - 1)(t - 1) + sum_{l in omega(t - 1)} (l - 1) automorphisms.
* The dual basis Omega_i^* of the power basis X^i for the pairing
  <P, Q> = Tr(P Q-bar), Q-bar(X) = Q(X^(M-1)), so that coefficient i of m is
  Tr(m Omega_i^*-bar) (Sec. 4.4), and Lemma 1's partial-trace rows.
* RnsRlwe: RLWE over the same ring modulo Q = prod q_i (q_i = 1 mod M), with
  encryption, decryption, key switching after an automorphism by the RNS
  limbs of tau_h(a), and the homomorphic tower trace (Sec. 2.1-2.3 on
  ciphertexts).
* TorusRlwe: the paper's own scheme, RLWE over the torus T_q, q = 2^53
  (Sec. 2.1), with the (D, l) gadget key switching of Sec. 2.2 / Sec. 4.2
  and Table 2, and the same homomorphic tower trace.
"""
from __future__ import annotations

import math
from fractions import Fraction


def prime_factors(x: int) -> list:
    """Prime factors of x with multiplicity (omega_x in Sec. 2.3)."""
    out, d = [], 2
    while d * d <= x:
        while x % d == 0:
            out.append(d)
            x //= d
        d += 1
    if x > 1:
        out.append(x)
    return out


class Ring:
    """K = Q[X] / Phi_M(X), M = t^alpha, elements as length-N coefficient lists
    (Python ints or Fractions)."""

    def __init__(self, t: int, alpha: int):
        assert prime_factors(t) == [t] and alpha >= 1
        self.t, self.alpha = t, alpha
        self.M = t ** alpha
        self.m = self.M // t                       # Phi_M(X) = Phi_t(X^m)
        self.N = (t - 1) * self.m                  # phi(M)

    # ---------------------------------------------------------- reduction
    def reduce(self, coeffs) -> list:
        """A polynomial of any degree -> its residue mod Phi_M: first mod
        X^M - 1 (Phi_M divides it), then every X^e with e >= N is replaced by
        -sum_{k < t-1} X^(e - N + k m)."""
        c = [0] * self.M
        for e, v in enumerate(coeffs):
            c[e % self.M] += v
        for e in range(self.M - 1, self.N - 1, -1):
            v = c[e]
            if v:
                c[e] = 0
                for k in range(self.t - 1):
                    c[e - self.N + k * self.m] -= v
        return c[:self.N]

    def monomial(self, e: int) -> list:
        """X^e (any integer e; X^M = 1)."""
        c = [0] * self.M
        c[e % self.M] = 1
        return self.reduce(c)

    # --------------------------------------------------------- arithmetic
    def add(self, a, b) -> list:
        return [x + y for x, y in zip(a, b)]

    def scale(self, a, c) -> list:
        return [c * x for x in a]

    def mul(self, a, b) -> list:
        """Schoolbook product, then reduction mod Phi_M."""
        prod = [0] * (len(a) + len(b) - 1)
        for i, x in enumerate(a):
            if x:
                for j, y in enumerate(b):
                    prod[i + j] += x * y
        return self.reduce(prod)

    def mod(self, a, q: int) -> list:
        return [x % q for x in a]

    # --------------------------------------------------------- Galois group
    def units(self) -> list:
        """(Z / MZ)^*: the automorphism indices d of Sec. 2.2."""
        return [d for d in range(1, self.M) if math.gcd(d, self.M) == 1]

    def automorphism(self, a, d: int) -> list:
        """tau_d(P) = P(X^d) mod Phi_M, gcd(d, M) = 1."""
        assert math.gcd(d, self.M) == 1
        c = [0] * self.M
        for i, v in enumerate(a):
            c[i * d % self.M] += v
        return self.reduce(c)

    def conj(self, a) -> list:
        """P-bar(X) = P(X^(M-1)) (Sec. 4.4)."""
        return self.automorphism(a, self.M - 1)

    def trace(self, a) -> list:
        """Tr(P) = sum over gcd(d, M) = 1 of P(X^d) mod Phi_M (Sec. 2.3, the definition)."""
        acc = [0] * self.N
        for d in self.units():
            acc = self.add(acc, self.automorphism(a, d))
        return acc

    def partial_trace(self, a, i: int) -> list:
        """Tr_{K / K_i}: the sum over Gal(K / K_i) = {d = 1 mod t^i} (by definition)."""
        acc = [0] * self.N
        for d in self.units():
            if d % (self.t ** i) == 1 % (self.t ** i):
                acc = self.add(acc, self.automorphism(a, d))
        return acc

    def primitive_root(self) -> int:
        """A generator of the cyclic group (Z / MZ)^* (t odd)."""
        assert self.t > 2
        n = self.N
        fac = sorted(set(prime_factors(n)))
        for g in range(2, self.M):
            if math.gcd(g, self.M) == 1 and all(pow(g, n // f, self.M) != 1 for f in fac):
                return g
        raise ValueError("no primitive root")

    def tower_steps(self, gamma: int = 0) -> list:
        """The steps (h, length) of the tower of Sec. 2.3 (t odd): each maps x
        to sum_{k < length} tau_h^k(x).  Tr_{K_(i+1) / K_i} for i = alpha - 1
        .. max(gamma, 1): the subgroup {d = 1 mod t^i} / {d = 1 mod t^(i+1)}
        is cyclic of order t, generated by 1 + t^i.  At gamma = 0 then
        Tr_{K_1 / K_0}: (Z / tZ)^* is cyclic of order t - 1, generated by a
        primitive root g mod M, taken one prime factor l of t - 1 at a time
        (the sum over a cyclic group of order n factors as
        prod_i sum_{j < l_i} g^(j n / (l_1 ... l_i))): h = g^rest acts on K_1
        with order l."""
        t, M = self.t, self.M
        steps = [((1 + t ** i) % M, t) for i in range(self.alpha - 1, max(gamma, 1) - 1, -1)]
        if gamma >= 1:
            return steps
        g = self.primitive_root()
        rest = t - 1
        for l in prime_factors(t - 1):
            rest //= l
            steps.append((pow(g, rest, M), l))
        return steps

    def tower_trace(self, a, gamma: int = 0, counter: list | None = None) -> list:
        """The full trace by the tower of Sec. 2.3 (t odd), or, with gamma >= 1,
        only Tr_{K / K_gamma} (the levels the server still computes when the
        client supplied Tr_{K_gamma / K_0}).  counter[0] is incremented once
        per automorphism (one key switch each on ciphertexts)."""
        x = list(a)
        for h, length in self.tower_steps(gamma):
            acc, cur = list(x), list(x)
            for _ in range(length - 1):
                cur = self.automorphism(cur, h)
                if counter is not None:
                    counter[0] += 1
                acc = self.add(acc, cur)
            x = acc
        return x

    def tower_ks_count(self, gamma: int = 0) -> int:
        """Automorphisms (key switches) of tower_trace: (alpha - 1)(t - 1)
        levels above K_1 (fewer when gamma > 1) plus sum (l - 1) over the
        prime factors of t - 1 when gamma = 0 (Sec. 2.3)."""
        top = (self.alpha - max(gamma, 1)) * (self.t - 1)
        return top + (sum(l - 1 for l in prime_factors(self.t - 1)) if gamma == 0 else 0)

    # --------------------------------------------------------- dual basis
    def trace_of_monomial(self, j: int) -> int:
        """Tr(X^j) by the definition (sum of the automorphisms of X^j), read at
        coefficient 0 (the trace of X^j is a rational constant)."""
        tr = self.trace(self.monomial(j))
        assert all(v == 0 for v in tr[1:])
        return tr[0]

    def dual_basis(self) -> list:
        """Omega_i^* for 0 <= i < N: Tr(X^k Omega_i^*-bar) = [k = i] for k < N.
        Written Omega_i^*-bar = sum_l c_l X^l, the condition is
        sum_l c_l Tr(X^(k + l)) = [k = i]: an N x N linear system in exact
        rationals (Gauss-Jordan).  Returns Omega_i^* (not its conjugate)."""
        N = self.N
        tr = [self.trace_of_monomial(j) for j in range(2 * N)]
        A = [[Fraction(tr[k + l]) for l in range(N)] for k in range(N)]
        inv = _invert(A)
        out = []
        for i in range(N):
            cbar = [inv[l][i] for l in range(N)]     # column i: solves A c = e_i
            out.append(self.conj(cbar))
        return out


def _invert(A):
    """Inverse of a square matrix of Fractions (Gauss-Jordan)."""
    n = len(A)
    M = [list(row) + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        p = M[col][col]
        M[col] = [v / p for v in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * b for a, b in zip(M[r], M[col])]
    return [row[n:] for row in M]


class RnsRlwe:
    """RLWE over K = Q[X]/Phi_M modulo Q = prod q_i (Sec. 2.1 at general t),
    residues per limb: a ciphertext is ([a mod q_i]_i, [b mod q_i]_i) with
    b = a s + m + e, the sign convention of the t = 2 scheme.  Key switching
    after an automorphism (Sec. 2.2) decomposes tau_h(a) by its RNS limbs,
    d_i = [tau_h(a)_i (Q/q_i)^-1]_{q_i}, so that tau_h(a) = sum_i d_i Q/q_i
    (mod Q), and uses one key pair per digit:
        kb_i = ka_i s + e_i + (Q/q_i) tau_h(s)  (mod Q).
    Then (a', b') = (-sum_i d_i ka_i, tau_h(b) - sum_i d_i kb_i) decrypts under
    s to tau_h(m) + tau_h(e) - sum_i d_i e_i.  Every product is the ring's
    exact product in Z[X]/Phi_M reduced mod q_j.  The uniform a, ka and the
    noise e are inputs (drawn by the caller)."""

    def __init__(self, ring: Ring, moduli):
        self.R = ring
        self.q = [int(x) for x in moduli]
        self.Q = 1
        for x in self.q:
            self.Q *= x

    def _mulq(self, a, b, q):
        return self.R.mod(self.R.mul(a, b), q)

    def residues(self, poly) -> list:
        """An integer polynomial (length N) as its L limbs."""
        return [[int(c) % q for c in poly] for q in self.q]

    def encrypt(self, s, a_res, m, e) -> tuple:
        """(a, b = a s + m + e) limb by limb; s, m, e integer polynomials."""
        b = []
        for j, q in enumerate(self.q):
            as_ = self._mulq(a_res[j], s, q)
            b.append([(x + int(mi) + int(ei)) % q for x, mi, ei in zip(as_, m, e)])
        return ([list(map(int, r)) for r in a_res], b)

    def decrypt(self, s, ct) -> list:
        """Residues of b - a s per limb (m + noise)."""
        a, b = ct
        return [[(y - x) % q for x, y in zip(self._mulq(a[j], s, q), b[j])] for j, q in enumerate(self.q)]

    def centered(self, res) -> list:
        """CRT of limb residues to the centered integer in (-Q/2, Q/2]."""
        out = []
        for k in range(len(res[0])):
            v = 0
            for j, q in enumerate(self.q):
                qh = self.Q // q
                v += res[j][k] * qh * pow(qh, -1, q)
            v %= self.Q
            out.append(v - self.Q if v > self.Q // 2 else v)
        return out

    def ksk(self, s, h: int, ka, e) -> list:
        """Key for tau_h: kb[i][j] = ka[i][j] s + e_i + (Q/q_i) tau_h(s) mod q_j;
        ka[i][j] uniform residues, e[i] integer noise polynomials."""
        ts = self.R.automorphism(list(s), h)
        kb = []
        for i, qi in enumerate(self.q):
            qh = self.Q // qi
            row = []
            for j, q in enumerate(self.q):
                prod = self._mulq(ka[i][j], s, q)
                row.append([(p + int(ei) + (qh % q) * x) % q for p, ei, x in zip(prod, e[i], ts)])
            kb.append(row)
        return kb

    def keyswitch(self, ct, h: int, ka, kb) -> tuple:
        """The automorphism tau_h of ct followed by the key switch back to s."""
        a, b = ct
        ta = [self.R.mod(self.R.automorphism(a[j], h), q) for j, q in enumerate(self.q)]
        tb = [self.R.mod(self.R.automorphism(b[j], h), q) for j, q in enumerate(self.q)]
        n = self.R.N
        a2 = [[0] * n for _ in self.q]
        b2 = [list(r) for r in tb]
        for i, qi in enumerate(self.q):
            w = pow(self.Q // qi, -1, qi)
            d = [(x * w) % qi for x in ta[i]]          # digit i, an integer polynomial in [0, q_i)
            for j, q in enumerate(self.q):
                pa = self._mulq(d, ka[i][j], q)
                pb = self._mulq(d, kb[i][j], q)
                a2[j] = [(x - y) % q for x, y in zip(a2[j], pa)]
                b2[j] = [(x - y) % q for x, y in zip(b2[j], pb)]
        return (a2, b2)

    def add(self, c1, c2) -> tuple:
        return tuple([[(x + y) % q for x, y in zip(u[j], v[j])] for j, q in enumerate(self.q)]
                     for u, v in zip(c1, c2))

    def hom_trace(self, ct, gamma: int, keys: dict, counter: list | None = None) -> tuple:
        """Tr_{K / K_gamma} (gamma >= 1) or the full trace (gamma = 0) on a
        ciphertext, along the tower's steps: x <- sum_{k < length} tau_h^k(x),
        every tau_h followed by its key switch; keys[h] = (ka, kb)."""
        x = ct
        for h, length in self.R.tower_steps(gamma):
            acc, cur = x, x
            for _ in range(length - 1):
                cur = self.keyswitch(cur, h, *keys[h])
                if counter is not None:
                    counter[0] += 1
                acc = self.add(acc, cur)
            x = acc
        return x


class TorusRlwe:
    """RLWE over the discrete torus T_q = (1/q) Z_q with q = 2^53 (Sec. 2.1) in
    the ring T_q[X]/Phi_M, with the gadget key switching of Sec. 2.2 and Sec.
    4.2: the key for tau_h is the l encryptions RLWE_s(tau_h(s) / D^i),
    i = 1 .. l, with the base D and depth l of Table 2.

    A torus value x / q is stored as the integer x in [0, q).  A ciphertext is
    (a, b) with b = a s + m + e (mod q), the convention of RnsRlwe.  The uniform
    a, ka and the noise e are inputs (drawn by the caller).

    * Products are taken of a torus polynomial and an integer polynomial
      (a digit polynomial or the secret): schoolbook in numpy uint64, i.e.
      modulo 2^64, which is exact modulo q because q divides 2^64, then the
      reduction mod Phi_M of Ring.reduce, then mod q.
    * Gadget decomposition of x in [0, q): xr = round(x D^l / q) mod D^l
      (halves rounded up), then the signed base-D digits d_1 .. d_l of xr,
      d_1 the most significant, each in [-floor(D/2), D - floor(D/2)), with
      sum_i d_i D^(l-i) = xr (mod D^l); so sum_i d_i / D^i equals x / q up to
      1 / (2 D^l) on the torus.  Digits are taken from the least significant
      end, a digit in the upper part of [0, D) becoming negative with a carry
      into the next one; the carry out of d_1 is dropped (a multiple of D^l,
      an integer on the torus).
    * The key message tau_h(s) / D^i is taken coefficient by coefficient as
      round(c q / D^i) mod q (halves rounded up).
    * Key switch after tau_h: with d_i the digit polynomials of tau_h(a),
      (a', b') = (-sum_i d_i ka_i, tau_h(b) - sum_i d_i kb_i) mod q, which
      decrypts to tau_h(m + e) - sum_i d_i e_i minus the gadget's rounding.
    """

    LOGQ = 53

    def __init__(self, ring: Ring, D: int, l: int):
        assert D >= 2 and l >= 1 and D ** l <= 2 ** self.LOGQ
        self.R, self.D, self.l = ring, int(D), int(l)
        self.q = 2 ** self.LOGQ

    # ------------------------------------------------------------ products
    def mul(self, a, b) -> list:
        """a b in Z_q[X]/Phi_M for integer polynomials a, b of length N (any
        signs): schoolbook modulo 2^64, reduction mod Phi_M, then mod q."""
        import numpy as np

        R = self.R
        A = np.array([int(x) % 2 ** 64 for x in a], dtype=np.uint64)
        B = np.array([int(x) % 2 ** 64 for x in b], dtype=np.uint64)
        prod = np.zeros(2 * R.N - 1, dtype=np.uint64)
        for i in np.nonzero(A)[0]:
            prod[i:i + R.N] += A[i] * B
        c = [0] * R.M
        for e, v in enumerate(prod.tolist()):
            c[e % R.M] += v
        return [v % self.q for v in R.reduce(c)]

    def add(self, c1, c2) -> tuple:
        return tuple([(x + y) % self.q for x, y in zip(u, v)] for u, v in zip(c1, c2))

    def centered(self, x) -> list:
        """Torus integers in [0, q) as representatives in [-q/2, q/2)."""
        h = self.q // 2
        return [(v + h) % self.q - h for v in x]

    # ------------------------------------------------------ enc, dec, codec
    def encode(self, mu, log_p: int) -> list:
        """mu in T_p, p = 2^log_p (integers mod p) -> the torus integers mu q / p."""
        return [(int(v) % 2 ** log_p) << (self.LOGQ - log_p) for v in mu]

    def decode(self, phase, log_p: int) -> list:
        """pi_p of Sec. 2.1: round(p x / q) mod p (halves rounded up)."""
        sh = self.LOGQ - log_p
        return [((v + (1 << (sh - 1))) >> sh) % 2 ** log_p for v in phase]

    def encrypt(self, s, a, m, e) -> tuple:
        """(a, b = a s + m + e mod q); a and m torus integers, s and e integer
        polynomials."""
        a = [int(x) % self.q for x in a]
        as_ = self.mul(a, s)
        return (a, [(x + int(mi) + int(ei)) % self.q for x, mi, ei in zip(as_, m, e)])

    def decrypt(self, s, ct) -> list:
        """The phase b - a s mod q (m + noise)."""
        a, b = ct
        return [(y - x) % self.q for x, y in zip(self.mul(a, s), b)]

    # --------------------------------------------------------------- gadget
    def decompose(self, x) -> list:
        """The l digit polynomials [d_1, .., d_l] of a torus polynomial x."""
        D, l, q = self.D, self.l, self.q
        Dl, half = D ** l, D // 2
        out = [[0] * len(x) for _ in range(l)]
        for k, v in enumerate(x):
            xr = ((int(v) % q) * Dl + q // 2) // q % Dl
            for i in range(l, 0, -1):
                r = xr % D
                xr //= D
                if r >= D - half:
                    r -= D
                    xr += 1
                out[i - 1][k] = r
        return out

    def gadget_message(self, c, i: int) -> list:
        """The torus polynomial c / D^i for an integer polynomial c:
        round(c_k q / D^i) mod q per coefficient."""
        Di = self.D ** i
        return [((2 * int(v) * self.q + Di) // (2 * Di)) % self.q for v in c]

    def ksk(self, s, h: int, ka, e) -> list:
        """kb_i = ka_i s + e_i + tau_h(s) / D^i (mod q), i = 1 .. l; ka[i - 1]
        uniform torus integers, e[i - 1] integer noise polynomials."""
        ts = self.R.automorphism(list(s), h)
        kb = []
        for i in range(1, self.l + 1):
            prod = self.mul(ka[i - 1], s)
            g = self.gadget_message(ts, i)
            kb.append([(p + int(ei) + gi) % self.q for p, ei, gi in zip(prod, e[i - 1], g)])
        return kb

    def keyswitch(self, ct, h: int, ka, kb) -> tuple:
        """tau_h of ct, then the gadget key switch back to s."""
        a, b = ct
        ta = [v % self.q for v in self.R.automorphism(list(a), h)]
        tb = [v % self.q for v in self.R.automorphism(list(b), h)]
        a2, b2 = [0] * self.R.N, tb
        for i, d in enumerate(self.decompose(ta)):
            pa, pb = self.mul(d, ka[i]), self.mul(d, kb[i])
            a2 = [(x - y) % self.q for x, y in zip(a2, pa)]
            b2 = [(x - y) % self.q for x, y in zip(b2, pb)]
        return (a2, b2)

    def hom_trace(self, ct, gamma: int, keys: dict, counter: list | None = None) -> tuple:
        """Tr_{K / K_gamma} (gamma >= 1) or the full trace (gamma = 0) on a
        torus ciphertext along the tower's steps: x <- sum_{k < length}
        tau_h^k(x), each tau_h followed by its key switch; keys[h] = (ka, kb)."""
        x = ct
        for h, length in self.R.tower_steps(gamma):
            acc, cur = x, x
            for _ in range(length - 1):
                cur = self.keyswitch(cur, h, *keys[h])
                if counter is not None:
                    counter[0] += 1
                acc = self.add(acc, cur)
            x = acc
        return x
