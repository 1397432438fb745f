"""Seeded synthetic workloads: parameter sets, layer shapes, float inputs and
weights.  Holds none of the method's arithmetic (no encoding, no modular
arithmetic); the GPU path and the CPU oracle both take their inputs from here.

Parameter sets (ring N = 2^log_n, L data primes + K special primes of the
given size, fixed-point scale Delta for inputs and weights):

* ``fc64``    N = 2^12, 2 x 30-bit + 1 special, Delta = 2^25: one 64x64 fully
  connected layer, W and x uniform in (-1, 1); 63 tree merges + 6 trace steps.
* ``conv16``  N = 2^14, 3 x 50-bit + 1 special, Delta = 2^40: one ResNet-20
  stage-1 convolution, 3x3, 16 -> 16 channels, pad 1, on a 16x32x32 input
  U(-1, 1), Kaiming-uniform weights U(+-sqrt(6/fan_in)); 16384 outputs packed
  into 2 ciphertexts of 8192 (16384 key switches).
* ``r18``     N = 2^15, 4 x 50-bit + 2 special (ResNet-18 on 3x64x64).
* ``r34``     N = 2^16, 5 x 50-bit + 2 special (ResNet-34 on 3x224x224).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class ParamSet:
    name: str
    log_n: int
    n_data: int
    data_bits: int
    n_special: int
    special_bits: int
    delta: float          # input and weight scale
    sigma: float = 3.2


PARAMS = {
    "fc64": ParamSet("fc64", 12, 2, 30, 1, 30, 2.0 ** 25),
    "conv16": ParamSet("conv16", 14, 3, 50, 1, 50, 2.0 ** 40),
    "r18": ParamSet("r18", 15, 4, 50, 2, 50, 2.0 ** 40),
    "r34": ParamSet("r34", 16, 5, 50, 2, 50, 2.0 ** 40),
}


@dataclass(frozen=True)
class Term:
    """A convolution over an input segment (mirrors sf_conv_term)."""
    in_offset: int
    H: int
    W: int
    C_in: int
    C_out: int
    kh: int
    kw: int
    stride: int = 1
    pad: int = 0

    @property
    def H_out(self):
        return (self.H + 2 * self.pad - self.kh) // self.stride + 1

    @property
    def W_out(self):
        return (self.W + 2 * self.pad - self.kw) // self.stride + 1

    @property
    def fan_in(self):
        return self.kh * self.kw * self.C_in


@dataclass
class LayerCase:
    name: str
    terms: list
    weights: list            # float64 per term [C_out][kh][kw][C_in]
    bias: np.ndarray | None
    x: np.ndarray            # float64 layer input, flattened (E_in values)
    sigma_prev: np.ndarray | None   # uint32[E_in]
    sigma_out: np.ndarray | None    # uint32[E_out]

    @property
    def E_in(self):
        return max(t.in_offset + t.H * t.W * t.C_in for t in self.terms)

    @property
    def E_out(self):
        t = self.terms[0]
        return t.H_out * t.W_out * t.C_out


def kaiming_uniform(rng, shape, fan_in):
    """He et al. 2015, gain sqrt(2): U(-sqrt(6/fan_in), sqrt(6/fan_in))."""
    b = np.sqrt(6.0 / fan_in)
    return rng.uniform(-b, b, shape)


def random_permutation(rng, n) -> np.ndarray:
    """A seeded permutation from numpy (stands in for a session's sigma)."""
    return rng.permutation(n).astype(np.uint32)


def fc64_case(seed: int = 101) -> LayerCase:
    rng = np.random.default_rng(seed)
    t = Term(0, 1, 1, 64, 64, 1, 1)
    W = rng.uniform(-1, 1, (64, 1, 1, 64))
    x = np.random.default_rng(seed + 1).uniform(-1, 1, 64)
    prng = np.random.default_rng(seed + 4)
    return LayerCase("fc64", [t], [W], None, x, random_permutation(prng, 64), random_permutation(prng, 64))


def conv16_case(seed: int = 201, shuffle: bool = True) -> LayerCase:
    rng = np.random.default_rng(seed)
    t = Term(0, 32, 32, 16, 16, 3, 3, 1, 1)
    W = kaiming_uniform(rng, (16, 3, 3, 16), t.fan_in)
    x = np.random.default_rng(seed + 1).uniform(-1, 1, 32 * 32 * 16)
    prng = np.random.default_rng(seed + 4)
    sp = random_permutation(prng, 32 * 32 * 16) if shuffle else None
    so = random_permutation(prng, 32 * 32 * 16) if shuffle else None
    return LayerCase("conv16", [t], [W], None, x, sp, so)


def small_conv_case(seed: int, H: int, W: int, C: int, Co: int, k: int = 3, stride: int = 1, pad: int = 1,
                    shortcut: bool = False, bias: bool = False, integer: bool = False, shuffle: bool = True,
                    x_range=(-1.0, 1.0)) -> LayerCase:
    """A scaled-down conv layer (optionally with a 1x1 strided shortcut term
    over a second input segment, and a bias), for full-chain parity tests."""
    rng = np.random.default_rng(seed)
    terms = [Term(0, H, W, C, Co, k, k, stride, pad)]
    if integer:
        ws = [rng.integers(-3, 4, (Co, k, k, C)).astype(np.float64)]
    else:
        ws = [kaiming_uniform(rng, (Co, k, k, C), k * k * C)]
    if shortcut:
        terms.append(Term(H * W * C, H, W, C, Co, 1, 1, stride, 0))
        ws.append(rng.integers(-2, 3, (Co, 1, 1, C)).astype(np.float64) if integer
                  else kaiming_uniform(rng, (Co, 1, 1, C), C))
    b = None
    if bias:
        b = rng.integers(-5, 6, Co).astype(np.float64) if integer else rng.uniform(-0.5, 0.5, Co)
    E_in = max(t.in_offset + t.H * t.W * t.C_in for t in terms)
    xr = np.random.default_rng(seed + 1)
    if integer:
        x = xr.integers(0, 16, E_in).astype(np.float64)
    else:
        x = xr.uniform(x_range[0], x_range[1], E_in)
    prng = np.random.default_rng(seed + 4)
    E_out = terms[0].H_out * terms[0].W_out * Co
    sp = random_permutation(prng, E_in) if shuffle else None
    so = random_permutation(prng, E_out) if shuffle else None
    return LayerCase(f"conv{H}x{W}x{C}->{Co}", terms, ws, b, x, sp, so)


def fc_case(seed: int, fan_in: int, fan_out: int, bias: bool = False, shuffle: bool = True) -> LayerCase:
    rng = np.random.default_rng(seed)
    t = Term(0, 1, 1, fan_in, fan_out, 1, 1)
    W = kaiming_uniform(rng, (fan_out, 1, 1, fan_in), fan_in)
    b = rng.uniform(-0.5, 0.5, fan_out) if bias else None
    x = np.random.default_rng(seed + 1).uniform(0, 1, fan_in)
    prng = np.random.default_rng(seed + 4)
    return LayerCase(f"fc{fan_in}->{fan_out}", [t], [W], b, x,
                     random_permutation(prng, fan_in) if shuffle else None,
                     random_permutation(prng, fan_out) if shuffle else None)


def float_reference(case: LayerCase) -> np.ndarray:
    """f(x) = A x + b in float64 (the plaintext layer), original output order."""
    t0 = case.terms[0]
    Ho, Wo, Co = t0.H_out, t0.W_out, t0.C_out
    y = np.zeros((Ho, Wo, Co))
    for t, w in zip(case.terms, case.weights):
        seg = case.x[t.in_offset:t.in_offset + t.H * t.W * t.C_in].reshape(t.H, t.W, t.C_in)
        pad = np.zeros((t.H + 2 * t.pad, t.W + 2 * t.pad, t.C_in))
        pad[t.pad:t.pad + t.H, t.pad:t.pad + t.W] = seg
        for dh in range(t.kh):
            for dw in range(t.kw):
                patch = pad[dh:dh + (Ho - 1) * t.stride + 1:t.stride, dw:dw + (Wo - 1) * t.stride + 1:t.stride]
                y += patch @ w[:, dh, dw, :].T
    if case.bias is not None:
        y += case.bias
    return y.ravel()


# ---------------------------------------------------------------------------
# ResNet-shaped networks as lists of layer rounds
# ---------------------------------------------------------------------------

@dataclass
class RoundSpec:
    """One server round: terms over named input tensors.

    inputs: names of the activation tensors concatenated (in order) into the
    round's flattened input; terms: (input index, Term with in_offset set)."""
    name: str
    inputs: list
    terms: list
    out: str
    relu: bool = True
    weights_seed: int = 0


def _term_over(k, H, W, C, Co, kh, stride, pad):
    return Term(k, H, W, C, Co, kh, kh, stride, pad)


NETS = {
    # image H (= W), image channels, stem (kernel, stride, channels), stage widths, blocks per stage, classes
    "resnet20": dict(H=32, C=3, stem=(3, 1, 16), stages=[16, 32, 64], blocks=[3, 3, 3], ncls=10, seed=1000),
    "resnet18": dict(H=64, C=3, stem=(3, 1, 64), stages=[64, 128, 256, 512], blocks=[2, 2, 2, 2], ncls=200,
                     seed=3000),
    "resnet34": dict(H=224, C=3, stem=(7, 2, 64), stages=[64, 128, 256, 512], blocks=[3, 4, 6, 3], ncls=1000,
                     seed=4000, pool=True),
    # small networks of the same structure, for tests
    "tiny_a": dict(H=8, C=2, stem=(3, 1, 4), stages=[4], blocks=[1], ncls=10, seed=5000),
    "tiny_b": dict(H=8, C=3, stem=(3, 1, 8), stages=[8, 8], blocks=[1, 1], ncls=5, seed=6000),
}


def resnet_rounds(kind: str) -> list:
    """Round lists of ResNet-shaped networks.  Batch norm is folded (identity
    on synthetic weights); ReLU runs on the client between rounds.  A basic
    block is two rounds; its second conv takes the block input as a second
    term (identity 1x1 for the same shape, 1x1 stride 2 to downsample).  The
    first block of every stage after the first has stride 2.  The global
    average pool is folded into the FC (a kernel as large as its input).

    resnet20: 3x32x32, 16/32/64 channels, 3 blocks per stage, FC 64 -> 10.
    resnet18: 3x64x64, 3x3 stem, no max-pool, 64/128/256/512, [2,2,2,2], FC -> 200.
    resnet34: 3x224x224, 7x7 stride-2 stem to 64x112x112; the 3x3 stride-2
      average pool is folded into the first block: its first conv becomes a
      7x7 stride-2 kernel over the stem output and its shortcut the pool itself
      (3x3 stride 2, per channel); [3,4,6,3] blocks, FC 512 -> 1000."""
    cfg = NETS[kind]
    seed = [cfg["seed"]]

    def nxt():
        seed[0] += 1
        return seed[0]

    sk, ss, sc_ = cfg["stem"]
    H0 = cfg["H"]
    rounds = [RoundSpec("stem", ["x"], [_term_over(0, H0, H0, cfg["C"], sc_, sk, ss, sk // 2)], "a0", True, nxt())]
    cur, cH, cC = "a0", (H0 + 2 * (sk // 2) - sk) // ss + 1, sc_
    for si, (Co, nb) in enumerate(zip(cfg["stages"], cfg["blocks"])):
        for bi in range(nb):
            pooled = cfg.get("pool", False) and si == 0 and bi == 0
            stride = 2 if (si > 0 and bi == 0) else 1
            mid, out = f"s{si}b{bi}m", f"s{si}b{bi}o"
            if pooled:
                oH = cH // 2
                t1 = _term_over(0, cH, cH, cC, Co, 7, 2, 3)
                sc = _term_over(oH * oH * Co, cH, cH, cC, Co, 3, 2, 1)
            else:
                oH = (cH - 1) // stride + 1
                t1 = _term_over(0, cH, cH, cC, Co, 3, stride, 1)
                sc = _term_over(oH * oH * Co, cH, cH, cC, Co, 1, stride, 0)
            rounds.append(RoundSpec(f"s{si}b{bi}c1", [cur], [t1], mid, True, nxt()))
            rounds.append(RoundSpec(f"s{si}b{bi}c2", [mid, cur], [_term_over(0, oH, oH, Co, Co, 3, 1, 1), sc],
                                    out, True, nxt()))
            cur, cH, cC = out, oH, Co
    rounds.append(RoundSpec("fc", [cur], [_term_over(0, cH, cH, cC, cfg["ncls"], cH, 1, 0)], "logits", False,
                            nxt()))
    return rounds


def network_input(kind: str, seed: int) -> np.ndarray:
    """A synthetic image for the network, U(0, 1), flattened (h, w, c)."""
    cfg = NETS[kind]
    return np.random.default_rng(seed).uniform(0.0, 1.0, cfg["H"] * cfg["H"] * cfg["C"])


def round_weights(spec: RoundSpec, integer: bool = False) -> list:
    """Seeded weights per term, [C_out][kh][kw][C_in]: Kaiming-uniform
    convolutions and downsampling shortcuts; the identity for a 1x1 stride-1
    shortcut; the 3x3 average (1/9 on the diagonal) for a pooled shortcut; the
    composition of a 3x3 conv with the 3x3 stride-2 average pool for the 7x7
    stride-2 kernel that follows it; and an FC weight spread evenly over the
    folded average pool.  ``integer``: small integers instead (exact mode)."""
    rng = np.random.default_rng(spec.weights_seed)
    ws = []
    for ti, t in enumerate(spec.terms):
        shape = (t.C_out, t.kh, t.kw, t.C_in)
        if integer:
            if ti == 1 and t.kh == 1 and t.stride == 1:
                w = np.zeros(shape)
                w[np.arange(t.C_out), 0, 0, np.arange(t.C_in)] = 1.0
            else:
                w = rng.integers(-2, 3, shape).astype(np.float64)
        elif ti == 1 and t.kh == 1 and t.stride == 1 and t.C_in == t.C_out:
            w = np.zeros(shape)
            w[np.arange(t.C_out), 0, 0, np.arange(t.C_in)] = 1.0
        elif ti == 1 and t.kh == 3:
            w = np.zeros(shape)
            w[np.arange(t.C_out), :, :, np.arange(t.C_in)] = 1.0 / 9.0
        elif spec.name == "fc":
            w = kaiming_uniform(rng, (t.C_out, 1, 1, t.C_in), t.C_in) / (t.kh * t.kw)
            w = np.broadcast_to(w, shape).copy()
        elif ti == 0 and t.kh == 7 and spec.name != "stem":
            w3 = kaiming_uniform(rng, (t.C_out, 3, 3, t.C_in), 9 * t.C_in)
            w = np.zeros(shape)
            for a in range(3):
                for e in range(3):
                    for b in range(3):
                        for f in range(3):
                            w[:, 2 * a + e, 2 * b + f, :] += w3[:, a, b, :] / 9.0
        else:
            w = kaiming_uniform(rng, shape, t.fan_in)
        ws.append(w)
    return ws


def round_input_size(spec: RoundSpec) -> int:
    return max(t.in_offset + t.H * t.W * t.C_in for t in spec.terms)


def round_output_size(spec: RoundSpec) -> int:
    t = spec.terms[0]
    return t.H_out * t.W_out * t.C_out


def round_case(kind: str, name: str, seed: int, shuffle: bool = True) -> LayerCase:
    """One round of a ResNet-shaped network as a stand-alone layer: the
    round's terms and seeded weights, an input U(0, 1) (a post-ReLU
    activation) and random input and output permutations."""
    spec = next(r for r in resnet_rounds(kind) if r.name == name)
    ws = round_weights(spec)
    e_in, e_out = round_input_size(spec), round_output_size(spec)
    x = np.random.default_rng(seed + 1).uniform(0.0, 1.0, e_in)
    prng = np.random.default_rng(seed + 4)
    sp = random_permutation(prng, e_in) if shuffle else None
    so = random_permutation(prng, e_out) if shuffle and spec.name != "fc" else None
    return LayerCase(f"{kind}.{name}", list(spec.terms), ws, None, x, sp, so)
