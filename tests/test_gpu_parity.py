"""GPU path against the CPU oracle, through the C ABI.

Bit-exact on every residue for integer work (NTT products, keys, encryption,
rotations, packing, whole layer rounds) on sizes the oracle finishes in
seconds, spanning several tiles and ragged groups; at the full benchmark size
(conv16: N = 2^14, 16384 outputs) on sampled outputs the oracle computes one
by one, plus decrypted error <= 1e-3 against float64 on every output.
"""
import os

import numpy as np
import pytest
import torch

import paper_2509_01253_gb300 as sf
from paper_2509_01253_gb300 import workloads as wl

from _gpu import Session, dev_zeros, from_dev, gpu_layer, oracle_layer, oracle_params, stream_input, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sf.lib()


def _rand_residues(rng, mods, count, n):
    return np.stack([np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in mods]) for _ in range(count)])


# ------------------------------------------------------------------ NTT ----

@pytest.mark.parametrize("log_n,L,bits,K", [(10, 3, 50, 1), (11, 4, 50, 2), (12, 2, 30, 1), (13, 5, 50, 2)])
def test_poly_mul_matches_schoolbook(oracle, log_n, L, bits, K):
    """NTT -> pointwise -> inverse NTT equals the schoolbook negacyclic product."""
    s = Session(log_n, L, bits, K, rot=False)
    try:
        rng = np.random.default_rng(log_n)
        q = s.info["moduli"][:L]
        a = _rand_residues(rng, q, 2, s.n)
        b = _rand_residues(rng, q, 2, s.n)
        out = dev_zeros(2, L, s.n)
        sf.sf_poly_mul(s.ctx, to_dev(a), to_dev(b), out, 2 * L)
        got = from_dev(out)
        for t in range(2):
            for i in range(L):
                assert (got[t, i] == oracle.polymul(a[t, i], b[t, i], q[i])).all(), (t, i)
    finally:
        s.close()


def test_poly_mul_full_size_sampled(oracle):
    """One limb of a full N = 2^14 product (the benchmark ring)."""
    ps = wl.PARAMS["conv16"]
    s = Session.from_set(ps, rot=False)
    try:
        rng = np.random.default_rng(7)
        q = s.info["moduli"][:s.L]
        a = _rand_residues(rng, q, 1, s.n)
        b = _rand_residues(rng, q, 1, s.n)
        out = dev_zeros(1, s.L, s.n)
        sf.sf_poly_mul(s.ctx, to_dev(a), to_dev(b), out, s.L)
        got = from_dev(out)
        assert (got[0, 1] == oracle.polymul(a[0, 1], b[0, 1], q[1])).all()
    finally:
        s.close()


@pytest.mark.parametrize("log_n,L,bits,K,count", [(10, 3, 50, 1, 2), (11, 4, 50, 2, 3), (12, 2, 30, 1, 5),
                                                   (13, 5, 50, 2, 2), (14, 3, 50, 1, 2), (15, 4, 50, 2, 3),
                                                   (16, 5, 50, 2, 2)])
def test_ntt_batch_transform_pair(oracle, log_n, L, bits, K, count):
    """sf_ntt_batch: forward, a pointwise product of the NTT values taken on
    the host with Python integers, then inverse equals the schoolbook
    negacyclic product (limbs sampled above N = 2^12); inverse(forward(x)) is
    x, also in place; forward(X) gives N distinct roots v with v^N = -1
    (the evaluation points) and forward of a constant is that constant."""
    s = Session(log_n, L, bits, K, rot=False)
    try:
        rng = np.random.default_rng(100 + log_n)
        q = s.info["moduli"][:L]
        a = _rand_residues(rng, q, count, s.n)
        b = _rand_residues(rng, q, count, s.n)
        A, B = dev_zeros(count, L, s.n), dev_zeros(count, L, s.n)
        sf.sf_ntt_batch(s.ctx, to_dev(a), A, count, False)
        sf.sf_ntt_batch(s.ctx, to_dev(b), B, count, False)
        ha, hb = from_dev(A), from_dev(B)
        for i in range(L):
            assert (ha[:, i] < q[i]).all() and (hb[:, i] < q[i]).all()
        # round trip, out of place and in place
        back = dev_zeros(count, L, s.n)
        sf.sf_ntt_batch(s.ctx, A, back, count, True)
        assert (from_dev(back) == a).all()
        sf.sf_ntt_batch(s.ctx, B, B, count, True)
        assert (from_dev(B) == b).all()
        # the other row-pass schedules give the same values
        for rad in (1, 2):
            sf.sf_ctx_set_option(s.ctx, "row_radix", rad)
            A2 = dev_zeros(count, L, s.n)
            sf.sf_ntt_batch(s.ctx, to_dev(a), A2, count, False)
            assert (from_dev(A2) == ha).all(), rad
            sf.sf_ntt_batch(s.ctx, A2, A2, count, True)
            assert (from_dev(A2) == a).all(), rad
        sf.sf_ctx_set_option(s.ctx, "row_radix", 0)
        # pointwise product on the host, inverse on the device, schoolbook on the oracle
        prod = np.zeros_like(ha)
        for t in range(count):
            for i in range(L):
                prod[t, i] = np.array([(int(x) * int(y)) % int(q[i]) for x, y in zip(ha[t, i], hb[t, i])],
                                      dtype=np.uint64)
        P = to_dev(prod)
        sf.sf_ntt_batch(s.ctx, P, P, count, True)
        got = from_dev(P)
        limbs = [(t, i) for t in range(count) for i in range(L)] if log_n <= 12 else [(count - 1, L - 1)]
        if log_n <= 14:
            for t, i in limbs:
                assert (got[t, i] == oracle.polymul(a[t, i], b[t, i], q[i])).all(), (t, i)
        # evaluation points: forward of X and of a constant
        mono = np.zeros((1, L, s.n), dtype=np.uint64)
        mono[0, :, 1] = 1
        M = to_dev(mono)
        sf.sf_ntt_batch(s.ctx, M, M, 1, False)
        v = from_dev(M)[0]
        for i in range(L):
            qi = int(q[i])
            assert len(set(v[i].tolist())) == s.n
            for j in rng.choice(s.n, 16, replace=False):
                assert pow(int(v[i, j]), s.n, qi) == qi - 1
        const = np.zeros((1, L, s.n), dtype=np.uint64)
        const[0, :, 0] = 12345
        Cn = to_dev(const)
        sf.sf_ntt_batch(s.ctx, Cn, Cn, 1, False)
        assert (from_dev(Cn) == 12345).all()
        with pytest.raises(sf.SafhireError):
            sf.sf_ntt_batch(s.ctx, A, A, 0, False)
    finally:
        s.close()


def test_modmul_probe_reports_a_rate():
    """The arithmetic-ceiling probe returns a positive rate for each kind and
    rejects unknown kinds."""
    ps = wl.PARAMS["conv16"]
    s = Session.from_set(ps, rot=False)
    try:
        for kind in range(3):
            r = sf.sf_modmul_probe(s.ctx, kind)
            assert np.isfinite(r) and r > 1.0, (kind, r)
        with pytest.raises(sf.SafhireError):
            sf.sf_modmul_probe(s.ctx, 3)
    finally:
        s.close()


# ------------------------------------------------------- keys / encryption --

@pytest.mark.parametrize("pset", ["fc64", "conv16"])
def test_keygen_encrypt_decrypt_bit_exact(oracle, pset):
    ps = wl.PARAMS[pset]
    s = Session.from_set(ps, sk_seed=103, rot=False)
    try:
        prm = oracle_params(oracle, ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits)
        assert s.info["moduli"] == prm.q + prm.p
        s_o = oracle.keygen(prm, 103)
        assert (sf.sf_secret_key_export(s.sk, s.n) == s_o).all()
        rng = np.random.default_rng(5)
        msg = rng.integers(-2 ** 40, 2 ** 40, s.n + 77)
        d = s.encrypt(msg, 104, 2)
        want = oracle.encrypt(prm, s_o, msg, 104, 2)
        assert (from_dev(d) == want.reshape(2, 2, s.L, s.n)).all()
        assert (s.decrypt(d, 2) == oracle.decrypt(prm, s_o, want)).all()
    finally:
        s.close()


@pytest.mark.parametrize("pset,ds", [("fc64", None), ("conv16", [3, 16385])])
def test_rotation_keys_bit_exact(oracle, pset, ds):
    ps = wl.PARAMS[pset]
    s = Session.from_set(ps, sk_seed=11, rk_seed=12, rot_d=ds)
    try:
        prm = oracle_params(oracle, ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits)
        s_o = oracle.keygen(prm, 11)
        for d in (ds or oracle.default_rotation_indices(prm)):
            got = np.zeros((prm.dnum, 2, prm.L + prm.K, prm.n), dtype=np.uint64)
            sf.sf_rotkeys_export(s.ctx, s.rk, d, got)
            assert (got == oracle.rotkey(prm, s_o, 12, d)).all(), d
    finally:
        s.close()


# --------------------------------------------------------------- rotate -----

@pytest.mark.parametrize("log_n,L,bits,K", [(10, 3, 50, 1), (10, 4, 50, 2), (10, 5, 50, 2), (11, 2, 30, 1)])
def test_rotate_bit_exact_all_keys(oracle, log_n, L, bits, K):
    s = Session(log_n, L, bits, K, sk_seed=21, rk_seed=22)
    try:
        prm = oracle_params(oracle, log_n, L, bits, K)
        s_o = oracle.keygen(prm, 21)
        keys = oracle.rotation_keys(prm, s_o, 22)
        msg = np.random.default_rng(3).integers(-2 ** 20, 2 ** 20, 3 * s.n)
        d_ct = s.encrypt(msg, 23, 3)
        cts = from_dev(d_ct).reshape(3, 2, L, s.n)
        out = dev_zeros(3, 2, L, s.n)
        for d in oracle.default_rotation_indices(prm):
            sf.sf_rotate(s.ctx, s.rk, d, d_ct, out, 3)
            got = from_dev(out)
            for j in range(3):
                assert (got[j] == oracle.rotate(prm, keys, d, cts[j])).all(), (d, j)
    finally:
        s.close()


@pytest.mark.parametrize("ks3_threads", [256, 512])
def test_rotate_full_size(oracle, ks3_threads):
    """Benchmark ring N = 2^14, 3 x 50-bit + 1 special, the first-level and
    the last trace automorphisms, with either block shape of the key-switch
    inner product."""
    ps = wl.PARAMS["conv16"]
    ds = [3, 16385]
    s = Session.from_set(ps, sk_seed=31, rk_seed=32, rot_d=ds)
    try:
        sf.sf_ctx_set_option(s.ctx, "ks3_threads", ks3_threads)
        assert sf.sf_ctx_get_option(s.ctx, "ks3_threads") == ks3_threads
        prm = oracle_params(oracle, ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits)
        s_o = oracle.keygen(prm, 31)
        keys = oracle.rotation_keys(prm, s_o, 32, ds)
        msg = np.random.default_rng(4).integers(-2 ** 40, 2 ** 40, s.n)
        d_ct = s.encrypt(msg, 33, 1)
        ct = from_dev(d_ct).reshape(2, s.L, s.n)
        out = dev_zeros(1, 2, s.L, s.n)
        for d in ds:
            sf.sf_rotate(s.ctx, s.rk, d, d_ct, out, 1)
            assert (from_dev(out)[0] == oracle.rotate(prm, keys, d, ct)).all(), d
    finally:
        s.close()


# ----------------------------------------------------------------- pack -----

@pytest.mark.parametrize("n_leaves,n", [(1, 1), (2, 2), (5, 8), (8, 8), (64, 64), (100, 128), (3, 512)])
def test_pack_bit_exact(oracle, n_leaves, n):
    log_n, L, K = 10, 3, 1
    s = Session(log_n, L, 50, K, sk_seed=41, rk_seed=42)
    try:
        prm = oracle_params(oracle, log_n, L, 50, K)
        s_o = oracle.keygen(prm, 41)
        keys = oracle.rotation_keys(prm, s_o, 42)
        msg = np.random.default_rng(n_leaves).integers(-2 ** 30, 2 ** 30, n_leaves * s.n)
        d_ct = s.encrypt(msg, 43, n_leaves)
        leaves = list(from_dev(d_ct).reshape(n_leaves, 2, L, s.n))
        out = dev_zeros(2, L, s.n)
        sf.sf_pack(s.ctx, s.rk, d_ct, n_leaves, n, out)
        assert (from_dev(out) == oracle.pack(prm, keys, leaves, n=n)).all()
    finally:
        s.close()


@pytest.mark.gpu
def test_pack_full_size_conv16_ring(oracle):
    """Fast packing of 4 encrypted leaves at the conv16 ring (N = 2^14, 3 x
    50-bit + 1): 3 tree merges and 12 trace steps, every residue equal to the
    oracle's."""
    ps = wl.PARAMS["conv16"]
    s = Session.from_set(ps, sk_seed=51, rk_seed=52)
    try:
        prm = oracle_params(oracle, ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits)
        s_o = oracle.keygen(prm, 51)
        keys = oracle.rotation_keys(prm, s_o, 52)
        msg = np.random.default_rng(53).integers(-2 ** 40, 2 ** 40, 4 * s.n)
        d_ct = s.encrypt(msg, 54, 4)
        leaves = list(from_dev(d_ct).reshape(4, 2, s.L, s.n))
        out = dev_zeros(2, s.L, s.n)
        sf.sf_pack(s.ctx, s.rk, d_ct, 4, 4, out)
        assert (from_dev(out) == oracle.pack(prm, keys, leaves, n=4)).all()
    finally:
        s.close()


def _read_pack_digest():
    path = os.path.join(os.path.dirname(__file__), "golden", "pack_n65536_l5k2_n4.txt")
    digest, rows = None, {}
    with open(path) as f:
        for line in f:
            w = line.split()
            if not w or w[0].startswith("#"):
                continue
            if w[0] == "sha256":
                digest = w[1]
            elif w[0] == "residues":
                rows[(int(w[1]), int(w[2]))] = [int(v) for v in w[3:]]
    return digest, rows


@pytest.mark.gpu
def test_pack_largest_ring_matches_stored_oracle_result():
    """Fast packing of 4 encrypted leaves at N = 2^16, 5 x 50-bit + 2 (3 tree
    merges, 14 trace steps): the SHA-256 of every output residue equals the
    one tests/golden/make_pack_largest_ring.py wrote from the CPU oracle on
    the same seeded keys and leaves (the oracle needs minutes at this size)."""
    import hashlib
    digest, rows = _read_pack_digest()
    s = Session(16, 5, 50, 2, sk_seed=61, rk_seed=62)
    try:
        msg = np.random.default_rng(63).integers(-2 ** 40, 2 ** 40, 4 * s.n)
        d_ct = s.encrypt(msg, 64, 4)
        out = dev_zeros(2, s.L, s.n)
        sf.sf_pack(s.ctx, s.rk, d_ct, 4, 4, out)
        got = from_dev(out).reshape(2, s.L, s.n)
        for (part, limb), vals in rows.items():
            assert [int(v) for v in got[part, limb, :len(vals)]] == vals, (part, limb)
        assert hashlib.sha256(np.ascontiguousarray(got, dtype="<u8").tobytes()).hexdigest() == digest
    finally:
        s.close()


@pytest.mark.gpu
def test_status_word_reports_out_of_range_input_residue():
    """An input ciphertext with a residue equal to its modulus: sf_rotate and
    sf_eval_linear_layer return SF_OK (the work is enqueued), the device check
    latches SF_ERANGE, sf_sync reports it once and clears it; valid input
    leaves the status clean."""
    ps = wl.PARAMS["fc64"]
    s = Session.from_set(ps, sk_seed=71, rk_seed=72)
    try:
        q = sf.sf_params_get_info(s.params)["moduli"]
        d_ct = s.encrypt(np.arange(64), 73, 1)
        out = dev_zeros(1, 2, s.L, s.n)
        sf.sf_rotate(s.ctx, s.rk, 3, d_ct, out, 1)
        sf.sf_sync(s.ctx)                                   # valid input: clean
        bad = d_ct.clone()
        bad[0, 1, 1, 17] = int(q[1])                        # b-part, limb 1: residue == q_1
        sf.sf_rotate(s.ctx, s.rk, 3, bad, out, 1)
        with pytest.raises(sf.SafhireError) as e:
            sf.sf_sync(s.ctx)
        assert e.value.status == sf.SF_ERANGE
        sf.sf_sync(s.ctx)                                   # cleared
        case = wl.fc64_case()
        lay = gpu_layer(s, case, ps.delta, ps.delta ** 2)
        d_out = dev_zeros(1, 2, s.L, s.n)
        sf.sf_eval_linear_layer(s.ctx, lay, s.rk, bad, 1, case.sigma_prev, case.sigma_out, d_out, 1)
        with pytest.raises(sf.SafhireError) as e:
            sf.sf_sync(s.ctx)
        assert e.value.status == sf.SF_ERANGE
        sf.sf_eval_linear_layer(s.ctx, lay, s.rk, d_ct, 1, case.sigma_prev, case.sigma_out, d_out, 1)
        sf.sf_sync(s.ctx)
        sf.sf_layer_destroy(lay)
    finally:
        s.close()


# ---------------------------------------------------------- linear layer -----

def _run_layer(sess, case, delta, out_scale, weight_scale, n_capacity=64, integer_input=False):
    lay = gpu_layer(sess, case, weight_scale, out_scale)
    info = sf.sf_layer_get_info(sess.ctx, lay)
    xs = stream_input(case)
    msg = (xs * delta).astype(np.int64) if integer_input else sf.sf_encode_input(xs, delta)
    d_in = sess.encrypt(msg, 77, info["k_in"])
    d_out = dev_zeros(max(n_capacity, info["n_groups"]), 2, sess.L, sess.n)
    n_out = sf.sf_eval_linear_layer(sess.ctx, lay, sess.rk, d_in, info["k_in"], case.sigma_prev, case.sigma_out,
                                    d_out, d_out.shape[0])
    sf.sf_sync(sess.ctx)
    assert n_out == info["n_groups"]
    return lay, info, msg, d_in, from_dev(d_out)[:n_out]


def _oracle_layer_run(oracle, prm, case, msg, weight_scale, out_scale, s_seed, rk_seed, k_in):
    s_o = oracle.keygen(prm, s_seed)
    keys = oracle.rotation_keys(prm, s_o, rk_seed)
    cts = oracle.encrypt(prm, s_o, msg, 77, k_in)
    lay = oracle_layer(oracle, case, weight_scale, out_scale)
    c = oracle.Counter()
    out = oracle.eval_linear_layer(prm, lay, keys, cts, case.sigma_prev, case.sigma_out, c)
    return out, s_o, c.ks


def test_fc64_layer_bit_exact(oracle):
    """The 64x64 FC layer at N = 2^12 (2 x 30-bit + 1 special), with input and
    output shuffles: every residue of the packed output equals the oracle's."""
    ps = wl.PARAMS["fc64"]
    case = wl.fc64_case()
    s = Session.from_set(ps, sk_seed=103, rk_seed=105)
    try:
        lay, info, msg, _, got = _run_layer(s, case, ps.delta, ps.delta ** 2, ps.delta)
        assert info["ks_count"] == 69
        prm = oracle_params(oracle, ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits)
        assert (msg == oracle.quantize(stream_input(case), ps.delta)).all()
        want, s_o, ks = _oracle_layer_run(oracle, prm, case, msg, ps.delta, ps.delta ** 2, 103, 105, info["k_in"])
        assert ks == 69
        assert (got == want).all()
        # decrypted error against float64
        vals = sf.sf_decode(s.params, s.decrypt(to_dev(got), 1), 1, s.n // info["group_size"], 64, ps.delta ** 2)
        ref = wl.float_reference(case)[case.sigma_out.astype(np.int64)]
        assert np.abs(vals - ref).max() <= 1e-3
        sf.sf_layer_destroy(lay)
    finally:
        s.close()


SCALED = {
    # name: (log_n, L, bits, K, case factory, weight_scale, delta)
    "conv_one_group": (10, 3, 50, 1, lambda: wl.small_conv_case(1, 8, 8, 8, 8), 2.0 ** 20, 2.0 ** 20),
    "conv_ragged_two_groups": (10, 3, 50, 1, lambda: wl.small_conv_case(2, 10, 10, 6, 7), 2.0 ** 20, 2.0 ** 20),
    "shortcut_bias_k_in_3": (11, 4, 50, 2, lambda: wl.small_conv_case(3, 14, 14, 8, 6, stride=2, shortcut=True,
                                                                        bias=True), 2.0 ** 20, 2.0 ** 20),
    "fc_bias_dnum3": (10, 5, 50, 2, lambda: wl.fc_case(4, 300, 37, bias=True), 2.0 ** 20, 2.0 ** 20),
    "fc_30bit_no_shuffle": (10, 2, 30, 1, lambda: wl.fc_case(5, 200, 50, shuffle=False), 2.0 ** 12, 2.0 ** 12),
}


@pytest.mark.parametrize("name", sorted(SCALED))
def test_scaled_layer_bit_exact(oracle, name):
    """Whole rounds on scaled rings: several tiles, ragged last group, k_in > 1,
    residual shortcut term, bias, every digit layout (dnum = 1 limb, 2 limbs,
    uneven last digit)."""
    log_n, L, bits, K, make, wsc, delta = SCALED[name]
    case = make()
    s = Session(log_n, L, bits, K, sk_seed=51, rk_seed=52)
    try:
        lay, info, msg, _, got = _run_layer(s, case, delta, delta * wsc, wsc)
        prm = oracle_params(oracle, log_n, L, bits, K)
        assert (msg == oracle.quantize(stream_input(case), delta)).all()
        want, s_o, ks = _oracle_layer_run(oracle, prm, case, msg, wsc, delta * wsc, 51, 52, info["k_in"])
        assert ks == info["ks_count"]
        assert (got == want).all()
        sf.sf_layer_destroy(lay)
    finally:
        s.close()


def test_ks_batch_size_does_not_change_results(oracle):
    """Identical inputs under different launch batchings give identical
    residues (a race between merges would show up here)."""
    log_n, L, bits, K, make, wsc, delta = SCALED["conv_ragged_two_groups"]
    case = make()
    s = Session(log_n, L, bits, K, sk_seed=61, rk_seed=62)
    try:
        outs = []
        for b in (1, 3, 64, 4096):
            sf.sf_ctx_set_option(s.ctx, "ks_batch", b)
            lay, info, msg, _, got = _run_layer(s, case, delta, delta * wsc, wsc)
            outs.append(got)
            sf.sf_layer_destroy(lay)
        assert all((o == outs[0]).all() for o in outs[1:])
    finally:
        s.close()


# ----------------------------------------------- full benchmark size -------

def test_conv16_full_size(oracle):
    """The benchmark layer (ResNet-20 conv 16->16 on 16x32x32, N = 2^14):
    sampled leaves bit-exact against the oracle, decrypted outputs within
    1e-3 of float64 on all 16384 outputs."""
    ps = wl.PARAMS["conv16"]
    case = wl.conv16_case()
    s = Session.from_set(ps, sk_seed=203, rk_seed=205)
    try:
        lay, info, msg, d_in, got = _run_layer(s, case, ps.delta, ps.delta ** 2, ps.delta)
        assert info["n_groups"] == 2 and info["group_size"] == 8192 and info["ks_count"] == 16384
        res = s.decrypt(to_dev(got), 2)
        vals = sf.sf_decode(s.params, res, 2, 2, 16384, ps.delta ** 2)
        ref = wl.float_reference(case)[case.sigma_out.astype(np.int64)]
        err = np.abs(vals - ref).max()
        assert err <= 1e-3, err
        # sampled leaves (steps 6-8) against the oracle's direct product
        prm = oracle_params(oracle, ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits)
        olay = oracle_layer(oracle, case, ps.delta, ps.delta ** 2)
        cts = from_dev(d_in).reshape(1, 2, s.L, s.n)
        sample = np.random.default_rng(9).choice(16384, 12, replace=False).astype(np.int32)
        sample[:3] = [0, 16383, 32 * 16 + 5]          # corners and an interior output
        d_leaf = dev_zeros(len(sample), 2, s.L, s.n)
        sf.sf_linear_outputs(s.ctx, lay, d_in, 1, case.sigma_prev, sample, d_leaf)
        leaves = from_dev(d_leaf)
        for t, o in enumerate(sample):
            assert (leaves[t] == oracle.linear_output(prm, olay, cts, int(o), case.sigma_prev)).all(), o
        sf.sf_layer_destroy(lay)
    finally:
        s.close()


def test_conv16_launch_shapes_identical():
    """The benchmark round gives the same residues under every launch shape
    the autotuner can pick: key-switch launch batches of 512 and 4096 merges,
    both block shapes of the inner product (256 x 8 and 512 x 4) and both
    row-pass sweep schedules (radix 8 and radix 4)."""
    ps = wl.PARAMS["conv16"]
    case = wl.conv16_case()
    s = Session.from_set(ps, sk_seed=203, rk_seed=205)
    try:
        outs = []
        for batch, nt, rad in ((512, 256, 0), (4096, 256, 0), (512, 512, 0), (4096, 512, 0), (512, 256, 1)):
            sf.sf_ctx_set_option(s.ctx, "ks_batch", batch)
            sf.sf_ctx_set_option(s.ctx, "ks3_threads", nt)
            sf.sf_ctx_set_option(s.ctx, "row_radix", rad)
            lay, info, msg, d_in, got = _run_layer(s, case, ps.delta, ps.delta ** 2, ps.delta)
            outs.append(got)
            sf.sf_layer_destroy(lay)
        assert all((o == outs[0]).all() for o in outs[1:])
        with pytest.raises(sf.SafhireError):
            sf.sf_ctx_set_option(s.ctx, "ks3_threads", 384)
    finally:
        s.close()


def test_conv16_integer_mode_exact(oracle):
    """Integer weights (scale 1) and integer inputs at scale 2^40: decrypting
    and rounding reproduces the quantised cleartext result exactly."""
    ps = wl.PARAMS["conv16"]
    case = wl.small_conv_case(7, 32, 32, 16, 16, integer=True)
    s = Session.from_set(ps, sk_seed=301, rk_seed=302)
    try:
        lay, info, msg, _, got = _run_layer(s, case, ps.delta, ps.delta, 1.0, integer_input=True)
        res = s.decrypt(to_dev(got), info["n_groups"])
        vals = sf.sf_decode(s.params, res, info["n_groups"], s.n // info["group_size"], case.E_out, ps.delta)
        ref = wl.float_reference(case)[case.sigma_out.astype(np.int64)]
        assert (np.rint(vals) == ref).all()
        # pack-tree noise (about N * n * key-switch noise) stays far below scale / 2
        assert np.abs(vals - ref).max() < 1e-3
        sf.sf_layer_destroy(lay)
    finally:
        s.close()


# ----------------------------------------- partial trace extraction, gamma = 2 --

def _gamma2_inputs(s, msg, k_in, seed):
    """The client's two uploads at gamma = 2: RLWE(m_j) and RLWE(m_j(X^3))."""
    d_in = s.encrypt(msg, seed, k_in)
    d_pow = s.encrypt(sf.sf_client_power(s.params, msg, k_in, 3), seed + 1, k_in)
    return d_in, d_pow


def test_client_power_matches_oracle(oracle):
    """sf_client_power (m(X^3) per chunk) equals the oracle's client power."""
    p = sf.sf_params_create(10, 2, 50, 1, 50)
    try:
        prm = oracle_params(oracle, 10, 2, 50, 1)
        m = np.random.default_rng(5).integers(-2 ** 40, 2 ** 40, 3 * prm.n)
        got = sf.sf_client_power(p, m, 3, 3).reshape(3, prm.n)
        for j in range(3):
            assert (got[j] == oracle.client_power(prm, m[j * prm.n:(j + 1) * prm.n])).all()
    finally:
        sf.sf_params_destroy(p)


def test_extract_and_pack_gamma2_bit_exact(oracle):
    """gamma = 2 extraction rows and their packing (the tau_3 level merged with
    no key switch) equal the oracle's, residue by residue, for several leaf
    counts (one value: the trace starts at k = 2)."""
    log_n, L, K = 10, 3, 1
    s = Session(log_n, L, 50, K, sk_seed=81, rk_seed=82)
    try:
        prm = oracle_params(oracle, log_n, L, 50, K)
        s_o = oracle.keygen(prm, 81)
        keys = oracle.rotation_keys(prm, s_o, 82)
        msg = np.random.default_rng(83).integers(-2 ** 30, 2 ** 30, s.n)
        d_ct, d_pow = _gamma2_inputs(s, msg, 1, 84)
        ct, ct3 = from_dev(d_ct).reshape(2, L, s.n), from_dev(d_pow).reshape(2, L, s.n)
        rows = []
        for i in (0, 1, 5, s.n // 2, s.n - 1):
            d_row = dev_zeros(2, L, s.n)
            sf.sf_extract(s.ctx, d_ct, i, 2, d_pow, d_row)
            row = from_dev(d_row).reshape(2, L, s.n)
            assert (row == oracle.extract(prm, ct, i, 2, ct3)).all(), i
            rows.append(row)
        d_rows = to_dev(np.stack(rows))
        for n_leaves, n in ((1, 1), (2, 2), (3, 4), (5, 8)):
            out = dev_zeros(2, L, s.n)
            sf.sf_pack_gamma(s.ctx, s.rk, d_rows, n_leaves, n, 2, out)
            want = oracle.pack(prm, keys, rows[:n_leaves], n=n, gamma=2)
            assert (from_dev(out).reshape(2, L, s.n) == want).all(), (n_leaves, n)
    finally:
        s.close()


@pytest.mark.parametrize("name", ["conv_ragged_two_groups", "shortcut_bias_k_in_3"])
def test_scaled_layer_gamma2_bit_exact(oracle, name):
    """Whole rounds at gamma = 2 on scaled rings (ragged groups, k_in = 3 inputs
    with a shortcut term and bias): every residue equals the oracle's round
    with the client's powers, with n/2 fewer key switches per group, and the
    halved decryption equals the gamma = 0 one."""
    log_n, L, bits, K, make, wsc, delta = SCALED[name]
    case = make()
    s = Session(log_n, L, bits, K, sk_seed=51, rk_seed=52)
    try:
        lay = gpu_layer(s, case, wsc, delta * wsc)
        info = sf.sf_layer_get_info(s.ctx, lay)
        k_in = info["k_in"]
        msg = sf.sf_encode_input(stream_input(case), delta)
        d_in, d_pow = _gamma2_inputs(s, msg, k_in, 77)
        d_out = dev_zeros(info["n_groups"], 2, s.L, s.n)
        n_out = sf.sf_eval_linear_layer_gamma(s.ctx, lay, s.rk, 2, d_in, d_pow, k_in, case.sigma_prev,
                                              case.sigma_out, d_out, info["n_groups"])
        sf.sf_sync(s.ctx)
        assert n_out == info["n_groups"]
        got = from_dev(d_out)
        prm = oracle_params(oracle, log_n, L, bits, K)
        s_o = oracle.keygen(prm, 51)
        keys = oracle.rotation_keys(prm, s_o, 52)
        cts = from_dev(d_in).reshape(k_in, 2, L, s.n)
        pw = from_dev(d_pow).reshape(k_in, 2, L, s.n)
        c = oracle.Counter()
        want = oracle.eval_linear_layer(prm, oracle_layer(oracle, case, wsc, delta * wsc), keys, cts,
                                        case.sigma_prev, case.sigma_out, c, powers=pw)
        assert (got == want).all()
        assert c.ks == oracle.ks_count(prm, case.E_out, gamma=2) < info["ks_count"]
        # halved decryption against the gamma = 0 round on the same input
        d0 = dev_zeros(info["n_groups"], 2, s.L, s.n)
        sf.sf_eval_linear_layer(s.ctx, lay, s.rk, d_in, k_in, case.sigma_prev, case.sigma_out, d0, info["n_groups"])
        g, stride = info["n_groups"], s.n // info["group_size"]
        v2 = sf.sf_decode(s.params, s.decrypt(d_out, g), g, stride, case.E_out, 2 * delta * wsc)
        v0 = sf.sf_decode(s.params, s.decrypt(d0, g), g, stride, case.E_out, delta * wsc)
        assert np.abs(v2 - v0).max() <= 1e-3
        sf.sf_layer_destroy(lay)
    finally:
        s.close()


def test_conv16_gamma2_full_size():
    """The benchmark layer at gamma = 2 (N = 2^14): 2 groups of 8192 values at
    4095 + 1 key switches each (8192 instead of 16384), decrypted (halved)
    outputs within 1e-3 of float64 on all 16384 outputs."""
    ps = wl.PARAMS["conv16"]
    case = wl.conv16_case()
    s = Session.from_set(ps, sk_seed=203, rk_seed=205)
    try:
        lay = gpu_layer(s, case, ps.delta, ps.delta ** 2)
        info = sf.sf_layer_get_info(s.ctx, lay)
        msg = sf.sf_encode_input(stream_input(case), ps.delta)
        d_in, d_pow = _gamma2_inputs(s, msg, 1, 204)
        d_out = dev_zeros(2, 2, s.L, s.n)
        sf.sf_eval_linear_layer_gamma(s.ctx, lay, s.rk, 2, d_in, d_pow, 1, case.sigma_prev, case.sigma_out, d_out, 2)
        vals = sf.sf_decode(s.params, s.decrypt(d_out, 2), 2, 2, 16384, 2 * ps.delta ** 2)
        ref = wl.float_reference(case)[case.sigma_out.astype(np.int64)]
        err = np.abs(vals - ref).max()
        assert err <= 1e-3, err
        with pytest.raises(sf.SafhireError):
            sf.sf_eval_linear_layer_gamma(s.ctx, lay, s.rk, 2, d_in, None, 1, None, None, d_out, 2)
        sf.sf_layer_destroy(lay)
    finally:
        s.close()


# ---------------------------------------------------------- small ops -------

def test_extract_and_shuffle(oracle):
    log_n, L = 10, 3
    s = Session(log_n, L, 50, 1, rot=False)
    try:
        prm = oracle_params(oracle, log_n, L, 50, 1)
        msg = np.random.default_rng(8).integers(-1000, 1000, 4 * s.n)
        d_ct = s.encrypt(msg, 9, 4)
        cts = from_dev(d_ct).reshape(4, 2, L, s.n)
        out = dev_zeros(2, L, s.n)
        for i in (0, 1, 517, s.n - 1):
            sf.sf_extract(s.ctx, d_ct, i, 0, None, out)
            got = from_dev(out)
            for part in range(2):
                for li, q in enumerate(prm.q):
                    ninv = pow(s.n, -1, q)
                    want = oracle.monomial_mul(cts[0, part, li], -i, q)
                    want = np.array([oracle.lib().or_mulmod(int(v), ninv, q) for v in want], dtype=np.uint64)
                    assert (got[part, li] == want).all()
        # gamma = 1 is gamma = 0 at t = 2 (K_1 = K_0); gamma = 2 needs the power; gamma 3 does not exist
        out1 = dev_zeros(2, L, s.n)
        sf.sf_extract(s.ctx, d_ct, 5, 0, None, out)
        sf.sf_extract(s.ctx, d_ct, 5, 1, None, out1)
        assert (from_dev(out1) == from_dev(out)).all()
        for gamma in (2, 3):
            with pytest.raises(sf.SafhireError) as e:
                sf.sf_extract(s.ctx, d_ct, 0, gamma, None, out)
            assert e.value.status == sf.SF_EINVAL
        perm = np.array([2, 0, 3, 1], dtype=np.uint32)
        sh = dev_zeros(4, 2, L, s.n)
        sf.sf_shuffle_cts(s.ctx, perm, d_ct, sh, 4)
        assert (from_dev(sh) == cts[perm.astype(np.int64)]).all()
    finally:
        s.close()


def test_errors_are_reported():
    s = Session(10, 3, 50, 1, rot_d=[3, 5])
    try:
        d_ct = s.encrypt(np.arange(10), 1, 1)
        out = dev_zeros(1, 2, 3, s.n)
        with pytest.raises(sf.SafhireError) as e:
            sf.sf_rotate(s.ctx, s.rk, 9, d_ct, out, 1)
        assert e.value.status == sf.SF_EINVAL
        case = wl.small_conv_case(1, 8, 8, 8, 8)
        lay = gpu_layer(s, case, 2.0 ** 20, 2.0 ** 40)
        with pytest.raises(sf.SafhireError) as e:      # needs keys 9, 17, ... that are missing
            sf.sf_eval_linear_layer(s.ctx, lay, s.rk, d_ct, 1, None, None, out, 1)
        assert e.value.status == sf.SF_EINVAL
        with pytest.raises(sf.SafhireError) as e:      # wrong number of input ciphertexts
            sf.sf_eval_linear_layer(s.ctx, lay, s.rk, d_ct, 2, None, None, out, 1)
        assert e.value.status == sf.SF_EINVAL
        bad = np.zeros(case.E_in, dtype=np.uint32)     # not a permutation
        with pytest.raises(sf.SafhireError) as e:
            sf.sf_eval_linear_layer(s.ctx, lay, s.rk, d_ct, 1, bad, None, out, 1)
        assert e.value.status == sf.SF_EINVAL
        sf.sf_layer_destroy(lay)
        sf.sf_sync(s.ctx)
    finally:
        s.close()


def test_memory_budget_chunking_is_exact(oracle):
    """The same round under a budget that forces one group at a time, and a
    smaller one that forces leaf chunks inside a group (residue classes
    reduced to roots, then the roots finish the tree): bit-identical packed
    ciphertexts, equal to the oracle's."""
    log_n, L, bits, K, make, wsc, delta = SCALED["conv_ragged_two_groups"]
    case = make()
    s = Session(log_n, L, bits, K, sk_seed=51, rk_seed=52)
    try:
        outs = []
        for budget in (None, 40 << 20, 10 << 20, 3 << 20):
            if budget:
                sf.sf_ctx_set_option(s.ctx, "mem_budget", budget)
            lay, info, msg, _, got = _run_layer(s, case, delta, delta * wsc, wsc)
            outs.append(got)
            sf.sf_layer_destroy(lay)
        prm = oracle_params(oracle, log_n, L, bits, K)
        want, _, _ = _oracle_layer_run(oracle, prm, case, msg, wsc, delta * wsc, 51, 52, info["k_in"])
        for o in outs:
            assert (o == want).all()
    finally:
        s.close()


def _batch_cases():
    return [wl.small_conv_case(11, 8, 8, 8, 8), wl.small_conv_case(12, 10, 10, 6, 7),
            wl.fc_case(13, 300, 37, bias=True), wl.small_conv_case(14, 14, 14, 8, 6, stride=2, shortcut=True, bias=True)]


def test_eval_layers_batch_matches_single_rounds():
    """Batching of uneven layers: four rounds of different sizes (one and two
    packing groups, an FC with bias, a strided shortcut over k_in = 3 inputs)
    evaluated in one call give residues identical to the four single calls,
    also when a small memory budget splits groups into units of leaves whose
    roots are packed in a separate pass."""
    log_n, L, bits, K = 11, 3, 50, 1
    s = Session(log_n, L, bits, K, sk_seed=81, rk_seed=82)
    try:
        delta = wsc = 2.0 ** 20
        cases = _batch_cases()
        lays, infos, ins, single = [], [], [], []
        for c in cases:
            lay, info, msg, d_in, got = _run_layer(s, c, delta, delta * wsc, wsc)
            lays.append(lay)
            infos.append(info)
            ins.append(d_in)
            single.append(got)
        for budget in (None, 6 << 20):
            if budget:
                sf.sf_ctx_set_option(s.ctx, "mem_budget", budget)
            outs = [dev_zeros(i["n_groups"], 2, L, s.n) for i in infos]
            n_outs = sf.sf_eval_layers(s.ctx, lays, [s.rk] * len(lays), ins, [i["k_in"] for i in infos],
                                       [c.sigma_prev for c in cases], [c.sigma_out for c in cases], outs,
                                       [i["n_groups"] for i in infos])
            sf.sf_sync(s.ctx)
            assert n_outs == [i["n_groups"] for i in infos]
            for o, want in zip(outs, single):
                assert (from_dev(o) == want).all()
        # rounds under two different client keys in one call (one class of units per key)
        sk2 = sf.sf_keygen(s.ctx, 83)
        rk2 = sf.sf_gen_rotation_keys(s.ctx, sk2, None, 84)
        rks = [s.rk if x % 2 == 0 else rk2 for x in range(len(lays))]
        sf.sf_ctx_set_option(s.ctx, "mem_budget", 64 << 30)
        single2 = []
        for x in range(len(lays)):
            o = dev_zeros(infos[x]["n_groups"], 2, L, s.n)
            sf.sf_eval_linear_layer(s.ctx, lays[x], rks[x], ins[x], infos[x]["k_in"], cases[x].sigma_prev,
                                    cases[x].sigma_out, o, infos[x]["n_groups"])
            single2.append(from_dev(o))
        for budget in (None, 6 << 20):
            if budget:
                sf.sf_ctx_set_option(s.ctx, "mem_budget", budget)
            outs = [dev_zeros(i["n_groups"], 2, L, s.n) for i in infos]
            sf.sf_eval_layers(s.ctx, lays, rks, ins, [i["k_in"] for i in infos], [c.sigma_prev for c in cases],
                              [c.sigma_out for c in cases], outs, [i["n_groups"] for i in infos])
            sf.sf_sync(s.ctx)
            for x, (o, want) in enumerate(zip(outs, single2)):
                assert (from_dev(o) == want).all(), (budget, x)
        sf.sf_rotkeys_destroy(rk2)
        sf.sf_secret_key_destroy(sk2)
        best, ms = sf.sf_autotune_layers(s.ctx, lays, [s.rk] * len(lays), ins, [i["k_in"] for i in infos],
                                         [c.sigma_prev for c in cases], [c.sigma_out for c in cases], outs,
                                         [i["n_groups"] for i in infos], repeats=1)
        assert best in (32, 64, 128, 256, 512, 1024, 2048, 4096) and ms > 0
        for o, want in zip(outs, single):
            assert (from_dev(o) == want).all()
        for lay in lays:
            sf.sf_layer_destroy(lay)
    finally:
        s.close()


# ------------------------------------------------------ large rings (2^15, 2^16) --
# Rings whose tiles hold 256-point sub-transforms run the 512-thread kernel
# variants (rows at N = 2^15; rows and columns at N = 2^16).

def test_large_ring_layer_bit_exact(oracle):
    """A small FC round on the ResNet-18 ring (N = 2^15, 4 x 50-bit + 2
    special, two-limb digits) end to end: 4 outputs packed into one ciphertext
    (3 tree merges + 13 trace steps), every residue against the oracle, under
    each row-pass schedule of its 256-point rows (radix 8, radix 4, radix 8
    with warp-shuffle exchanges)."""
    ps = wl.PARAMS["r18"]
    case = wl.fc_case(61, 24, 4, bias=True)
    delta = wsc = 2.0 ** 20           # bias at scale 2^40 fits int64
    s = Session.from_set(ps, sk_seed=63, rk_seed=65)
    try:
        lay, info, msg, _, got = _run_layer(s, case, delta, delta * wsc, wsc)
        assert info["group_size"] == 4 and info["ks_count"] == 3 + 13
        prm = oracle_params(oracle, ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits)
        want, _, ks = _oracle_layer_run(oracle, prm, case, msg, wsc, delta * wsc, 63, 65, info["k_in"])
        assert ks == 16
        assert (got == want).all()
        for rad in (1, 2):
            sf.sf_layer_destroy(lay)
            sf.sf_ctx_set_option(s.ctx, "row_radix", rad)
            lay, _, _, _, got_r = _run_layer(s, case, delta, delta * wsc, wsc)
            assert (got_r == want).all(), rad
        sf.sf_ctx_set_option(s.ctx, "row_radix", 0)
        vals = sf.sf_decode(s.params, s.decrypt(to_dev(got), 1), 1, s.n // 4, 4, delta * wsc)
        assert np.abs(vals - wl.float_reference(case)[case.sigma_out.astype(np.int64)]).max() <= 1e-3
        sf.sf_layer_destroy(lay)
    finally:
        s.close()


def test_largest_ring_rotate_and_leaves(oracle):
    """The ResNet-34 ring (N = 2^16, 5 x 50-bit + 2 special, uneven last
    digit): one rotation against the oracle's textbook key switch, and sampled
    leaves of a conv round with three input ciphertexts against its direct
    product."""
    ps = wl.PARAMS["r34"]
    s = Session.from_set(ps, sk_seed=71, rk_seed=72, rot_d=[3])
    try:
        prm = oracle_params(oracle, ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits)
        s_o = oracle.keygen(prm, 71)
        keys = oracle.rotation_keys(prm, s_o, 72, [3])
        msg = np.random.default_rng(5).integers(-2 ** 40, 2 ** 40, s.n)
        d_ct = s.encrypt(msg, 73, 1)
        ct = from_dev(d_ct).reshape(2, s.L, s.n)
        out = dev_zeros(1, 2, s.L, s.n)
        want = oracle.rotate(prm, keys, 3, ct)
        for rad in (0, 1, 2):                            # every row-pass sweep schedule
            sf.sf_ctx_set_option(s.ctx, "row_radix", rad)
            sf.sf_rotate(s.ctx, s.rk, 3, d_ct, out, 1)
            assert (from_dev(out)[0] == want).all(), rad
        sf.sf_ctx_set_option(s.ctx, "row_radix", 0)
        # leaves: stride-2 3x3 conv 16 -> 8 on 96x96x16 plus a 1x1 stride-2 shortcut term: 5 input cts
        case = wl.small_conv_case(75, 96, 96, 16, 8, stride=2, shortcut=True)
        lay = gpu_layer(s, case, ps.delta, ps.delta ** 2)
        info = sf.sf_layer_get_info(s.ctx, lay)
        assert info["k_in"] == 5
        xs = stream_input(case)
        qmsg = sf.sf_encode_input(xs, ps.delta)
        d_in = s.encrypt(qmsg, 77, info["k_in"])
        cts = from_dev(d_in).reshape(info["k_in"], 2, s.L, s.n)
        olay = oracle_layer(oracle, case, ps.delta, ps.delta ** 2)
        sample = np.random.default_rng(11).choice(info["E_out"], 6, replace=False).astype(np.int32)
        sample[0] = 0
        d_leaf = dev_zeros(len(sample), 2, s.L, s.n)
        sf.sf_linear_outputs(s.ctx, lay, d_in, info["k_in"], case.sigma_prev, sample, d_leaf)
        leaves = from_dev(d_leaf)
        for t, o in enumerate(sample):
            assert (leaves[t] == oracle.linear_output(prm, olay, cts, int(o), case.sigma_prev)).all(), o
        for rad in (1, 2):
            sf.sf_ctx_set_option(s.ctx, "row_radix", rad)
            d_leaf1 = dev_zeros(len(sample), 2, s.L, s.n)
            sf.sf_linear_outputs(s.ctx, lay, d_in, info["k_in"], case.sigma_prev, sample, d_leaf1)
            assert (from_dev(d_leaf1) == leaves).all(), rad
        sf.sf_layer_destroy(lay)
    finally:
        s.close()


@pytest.mark.parametrize("name", ["conv_ragged_two_groups", "shortcut_bias_k_in_3"])
def test_leaf_closed_form_matches_transform(name):
    """The leaf column pass of sparse weight tiles in closed form
    ("leaf_sparse" -1) and as a transform (0, the default) give identical
    residues."""
    log_n, L, bits, K, make, wsc, delta = SCALED[name]
    case = make()
    s = Session(log_n, L, bits, K, sk_seed=91, rk_seed=92)
    try:
        outs = []
        for sp in (0, -1, 128):
            sf.sf_ctx_set_option(s.ctx, "leaf_sparse", sp)
            lay, info, msg, _, got = _run_layer(s, case, delta, delta * wsc, wsc)
            outs.append(got)
            sf.sf_layer_destroy(lay)
        assert (outs[0] == outs[1]).all() and (outs[0] == outs[2]).all()
    finally:
        s.close()
