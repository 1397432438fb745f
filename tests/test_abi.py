"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point declared in include/safhire.h; host-side logic (parameters,
permutations, encoding, CRT decoding, argument validation) agrees with the
oracle and rejects bad input."""
import os
import re

import numpy as np
import pytest

import paper_2509_01253_gb300 as sf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    with open(os.path.join(ROOT, "include", "safhire.h")) as f:
        text = f.read()
    for m in re.finditer(r"^\s*(?:sf_status|void|const char \*)\s*(sf_\w+)\s*\(", text, re.M):
        names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported_and_bound():
    lib = sf.lib()
    declared = _declared()
    assert len(declared) >= 30
    for name in declared:
        assert hasattr(lib, name), name
        assert name in sf.EXPORTED, f"{name} has no Python binding"
    assert sf.sf_version().startswith("safhire-gb300")


def test_library_is_the_in_tree_build():
    assert os.path.dirname(sf.library_path()) == os.path.join(ROOT, "paper_2509_01253_gb300")
    assert os.path.exists(sf.library_path())


@pytest.mark.parametrize("log_n,L,bits,K", [(12, 2, 30, 1), (14, 3, 50, 1), (15, 4, 50, 2), (16, 5, 50, 2)])
def test_params_primes_match_oracle(oracle, log_n, L, bits, K):
    p = sf.sf_params_create(log_n, L, bits, K, bits)
    try:
        info = sf.sf_params_get_info(p)
        prm = oracle.make_params(log_n, L, bits, K, bits)
        assert info["moduli"] == prm.q + prm.p
        assert info["dnum"] == prm.dnum and info["n"] == prm.n
    finally:
        sf.sf_params_destroy(p)


def test_params_reject_bad_values():
    for args in [(9, 3, 50, 1, 50), (17, 3, 50, 1, 50), (14, 0, 50, 1, 50), (14, 3, 51, 1, 50),
                 (14, 3, 50, 5, 50), (14, 11, 50, 2, 50)]:
        with pytest.raises(sf.SafhireError) as e:
            sf.sf_params_create(*args)
        assert e.value.status == sf.SF_EINVAL


@pytest.mark.parametrize("seed,rnd,n", [(105, 1, 64), (105, 2, 64), (7, 3, 16384), (1, 0, 1), (2, 5, 2)])
def test_permutation_matches_oracle(oracle, seed, rnd, n):
    assert (sf.sf_permutation(seed, rnd, n) == oracle.permutation(seed, rnd, n)).all()


def test_encode_input_matches_oracle(oracle):
    x = np.random.default_rng(1).uniform(-1, 1, 10000)
    x[:4] = [0.5 / 2 ** 25, -0.5 / 2 ** 25, 1.5 / 2 ** 25, 0.0]
    assert (sf.sf_encode_input(x, 2.0 ** 25) == oracle.quantize(x, 2.0 ** 25)).all()
    with pytest.raises(sf.SafhireError) as e:
        sf.sf_encode_input(np.array([1e30]), 1.0)
    assert e.value.status == sf.SF_ERANGE


@pytest.mark.parametrize("log_n,L,bits,K", [(12, 2, 30, 1), (14, 3, 50, 1), (16, 5, 50, 2)])
def test_decode_matches_big_integer_crt(oracle, log_n, L, bits, K):
    """sf_decode (mixed-radix CRT, centring, division) against Python ints."""
    p = sf.sf_params_create(log_n, L, bits, K, bits)
    try:
        prm = oracle.make_params(log_n, L, bits, K, bits)
        n = prm.n
        rng = np.random.default_rng(log_n)
        Q = prm.Q
        lim = Q // 4
        vals = [int(v) % lim * (1 if v > 0 else -1) for v in rng.integers(-2 ** 62, 2 ** 62, 64)]
        vals += [0, 1, -1, (Q - 1) // 2, -((Q - 1) // 2)]
        vals += [(int(rng.integers(0, 2 ** 62)) * 2 ** 40 % lim) * (1 if i % 2 else -1) for i in range(16)]
        res = np.zeros((1, L, n), dtype=np.uint64)
        for k, v in enumerate(vals):
            for i, q in enumerate(prm.q):
                res[0, i, k] = v % q
        scale = 2.0 ** 37
        got = sf.sf_decode(p, res, 1, 1, len(vals), scale)
        want = np.array([v / scale for v in vals])
        assert np.allclose(got, want, rtol=1e-15, atol=0)
        # stride read-out: value v at coefficient (v mod (N/stride)) * stride of ct v // (N/stride)
        got2 = sf.sf_decode(p, res, 1, n // 2, 2, 1.0)
        assert got2[0] == vals[0] and got2[1] == 0.0
        with pytest.raises(sf.SafhireError):
            sf.sf_decode(p, res, 1, 3, 1, 1.0)
    finally:
        sf.sf_params_destroy(p)


def test_device_calls_fail_loudly_without_gpu():
    """With no usable CUDA device the context cannot be created: there is no
    CPU fallback."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = sf.sf_params_create(12, 2, 30, 1, 30)
    try:
        with pytest.raises(sf.SafhireError) as e:
            sf.sf_ctx_create(p, 0)
        assert e.value.status == sf.SF_ECUDA
    finally:
        sf.sf_params_destroy(p)
