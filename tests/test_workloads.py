"""Host logic of the network workloads (no GPU): the round lists of the
benchmark networks against the output and key-switch totals of the paper's
algorithm at t = 2 (n = min(N/2, next power of two >= E') per group,
(n - 1) + log2(N/n) key switches per group), the shapes that chain one round
into the next, and the client-side bookkeeping of inputs and permutations."""
import math

import numpy as np
import pytest

from paper_2509_01253_gb300 import workloads as wl


def _ks(E, N):
    n = min(N // 2, 1 << max(0, (E - 1).bit_length()))
    groups = -(-E // n)
    return groups * ((n - 1) + int(math.log2(N // n)))


@pytest.mark.parametrize("kind,N,rounds,outputs,ks", [
    ("resnet20", 2 ** 14, 20, 188_426, 188_447),
    ("resnet18", 2 ** 15, 18, 2_228_424, 2_228_486),
    ("resnet34", 2 ** 16, 34, 3_563_496, None),
])
def test_round_list_totals(kind, N, rounds, outputs, ks):
    rs = wl.resnet_rounds(kind)
    assert len(rs) == rounds
    assert sum(wl.round_output_size(r) for r in rs) == outputs
    if ks is not None:
        assert sum(_ks(wl.round_output_size(r), N) for r in rs) == ks


@pytest.mark.parametrize("kind", ["resnet20", "resnet18", "resnet34", "tiny_a", "tiny_b"])
def test_rounds_chain(kind):
    """Every round reads tensors produced earlier, and each term reads exactly
    its own segment of the concatenated input."""
    rs = wl.resnet_rounds(kind)
    sizes = {"x": wl.NETS[kind]["H"] ** 2 * wl.NETS[kind]["C"]}
    for r in rs:
        off = 0
        for name, t in zip(r.inputs, r.terms):
            assert name in sizes, (r.name, name)
            assert t.in_offset == off
            assert t.H * t.W * t.C_in == sizes[name]
            off += sizes[name]
        assert wl.round_input_size(r) == off
        shapes = {(t.H_out, t.W_out, t.C_out) for t in r.terms}
        assert len(shapes) == 1, r.name        # all terms land on the same output
        sizes[r.out] = wl.round_output_size(r)
    assert not rs[-1].relu and all(r.relu for r in rs[:-1])


def test_resnet34_pool_folding():
    """The 3x3 stride-2 average pool after the stem is folded into the first
    block: a 7x7 stride-2 conv with 7 x 7 x 64 = 3136 taps, and a pooled
    shortcut whose weights are the 3x3 average on the diagonal."""
    rs = wl.resnet_rounds("resnet34")
    c1, c2 = rs[1], rs[2]
    t = c1.terms[0]
    assert (t.kh, t.stride, t.pad, t.H, t.H_out) == (7, 2, 3, 112, 56)
    assert t.kh * t.kw * t.C_in == 3136
    sc = c2.terms[1]
    assert (sc.kh, sc.stride, sc.pad, sc.H, sc.H_out) == (3, 2, 1, 112, 56)
    w = wl.round_weights(c2)[1]
    assert np.allclose(w[np.arange(64), :, :, np.arange(64)], 1.0 / 9.0)
    w[np.arange(64), :, :, np.arange(64)] = 0.0
    assert not w.any()


def test_folded_kernel_is_conv_of_pool():
    """The 7x7 stride-2 weights equal the 3x3 conv applied after the 3x3
    stride-2 average pool (away from the image border)."""
    rs = wl.resnet_rounds("resnet34")
    spec = rs[1]
    W7 = wl.round_weights(spec)[0]
    rng = np.random.default_rng(spec.weights_seed)
    W3 = wl.kaiming_uniform(rng, (64, 3, 3, 64), 9 * 64)
    x = np.random.default_rng(0).uniform(0, 1, (15, 15, 64))
    # pooled map p[u] = mean of x[2u-1 .. 2u+1]; conv3 output at (i, j) reads p[i-1 .. i+1]
    i = j = 3
    p = lambda u, v: x[2 * u - 1:2 * u + 2, 2 * v - 1:2 * v + 2].mean(axis=(0, 1))
    want = sum(W3[:, a, b, :] @ p(i - 1 + a, j - 1 + b) for a in range(3) for b in range(3))
    got = sum(W7[:, dh, dw, :] @ x[2 * i - 3 + dh, 2 * j - 3 + dw] for dh in range(7) for dw in range(7))
    assert np.allclose(got, want)


def test_identity_shortcut_weights():
    spec = wl.resnet_rounds("resnet20")[2]          # s0b0c2: 16 -> 16, stride 1
    w = wl.round_weights(spec)[1]
    assert w.shape == (16, 1, 1, 16) and np.array_equal(w[:, 0, 0, :], np.eye(16))


class _Net:
    """Stands in for an encoded network (rounds and their sizes only)."""

    def __init__(self, kind):
        self.rounds = wl.resnet_rounds(kind)
        self.infos = [{"E_in": wl.round_input_size(r), "E_out": wl.round_output_size(r)} for r in self.rounds]

        class _PS:
            delta = 2.0 ** 20
        self.ps = _PS()
        self.quant = False


def test_client_concatenates_inputs_and_permutations():
    from paper_2509_01253_gb300 import network as nw
    net = _Net("tiny_a")
    x = np.arange(wl.NETS["tiny_a"]["H"] ** 2 * wl.NETS["tiny_a"]["C"], dtype=np.float64)
    c = nw.ClientState(net, x, session_seed=5, request_seed=6)
    stream, sigma = c.round_input(0)
    assert sigma is None and np.array_equal(stream, x)
    # round 0 output arrives in the order of a permutation: slot k holds y[perm[k]]
    E0 = net.infos[0]["E_out"]
    perm0 = np.random.default_rng(1).permutation(E0).astype(np.uint32)
    y0 = np.linspace(-1, 1, E0)
    c.absorb(0, y0[perm0], perm0)
    assert c.round == 1
    # ReLU on the shuffled values, kept in stream order with their permutation
    v, p = c.acts["a0"]
    assert np.array_equal(v, np.maximum(y0[perm0], 0)) and np.array_equal(p, perm0)
    # round 1 reads a0 only; round 2 reads [round-1 output, a0]: concatenated, offsets added
    perm1 = np.random.default_rng(2).permutation(E0).astype(np.uint32)
    y1 = np.linspace(0, 2, E0)
    c.absorb(1, y1[perm1], perm1)
    stream, sigma = c.round_input(2)
    assert np.array_equal(sigma[:E0], perm1) and np.array_equal(sigma[E0:], perm0.astype(np.int64) + E0)
    # unshuffling the stream gives the original-order concatenation
    orig = c.original_order(stream, sigma)
    assert np.array_equal(orig[:E0], np.maximum(y1, 0)) and np.array_equal(orig[E0:], np.maximum(y0, 0))


def test_requantisation_rule():
    """Sec. 4.5: after ReLU, y -> clip(round(y / eta), 0, 2^bits - 1), rounding
    half away from zero; eta is 2^floor(log2 fan_in) of the round."""
    from paper_2509_01253_gb300 import network as nw
    y = np.array([-5.0, 0.0, 5.0, 6.0, 9.0, 10.0, 100.0])
    assert nw.requantize(np.maximum(y, 0), 4, 4).tolist() == [0, 0, 1, 2, 2, 3, 15]
    assert nw.round_half_away(np.array([-2.5, -1.5, -0.4, 0.5, 1.5, 2.49])).tolist() == [-3, -2, 0, 1, 2, 2]
    rounds = wl.resnet_rounds("tiny_a")
    fans = [sum(t.kh * t.kw * t.C_in for t in r.terms) for r in rounds]
    assert fans[0] == 18 and nw.requant_scale(rounds[0]) == 16
    for r, f in zip(rounds, fans):
        e = nw.requant_scale(r)
        assert e <= f < 2 * e and (e & (e - 1)) == 0


def test_quantised_client_encodes_integers_and_requantises():
    """Quantised client: the image becomes 4-bit integers, a round's message is
    the integer stream times Delta exactly, and decoded outputs are rounded,
    passed through ReLU and requantised with the round's eta (the FC's
    outputs are kept as integer logits)."""
    from paper_2509_01253_gb300 import network as nw
    net = _Net("tiny_a")
    net.quant, net.act_bits = True, 4
    net.etas = [nw.requant_scale(r) for r in net.rounds]
    x = np.linspace(0.0, 1.0, wl.NETS["tiny_a"]["H"] ** 2 * wl.NETS["tiny_a"]["C"])
    c = nw.ClientState(net, x, session_seed=5, request_seed=6)
    xq = c.acts["x"][0]
    assert xq.min() == 0 and xq.max() == 15 and np.array_equal(xq, np.floor(x * 15 + 0.5))
    msg, sigma, stream = c.encode(0)
    assert sigma is None and msg.dtype == np.int64 and np.array_equal(msg, xq.astype(np.int64) * 2 ** 20)
    E0 = net.infos[0]["E_out"]
    y = np.arange(E0, dtype=np.float64) - E0 / 2 + 0.2        # decoded values: integers plus decoding error
    c.absorb(0, y, None)
    want = np.clip(np.floor(np.maximum(np.floor(y + 0.5), 0) / net.etas[0] + 0.5), 0, 15)
    assert np.array_equal(c.acts["a0"][0], want)
    # the last round (FC, no ReLU) keeps rounded integer logits
    last = len(net.rounds) - 1
    c.round = last
    logits = np.array([-3.2, 7.9, 0.4])
    c.absorb(last, logits, None)
    assert c.logits().tolist() == [-3, 8, 0]
