"""Encrypted inference over a network's rounds (Sec. 4.4 protocol, t = 2,
gamma = 0), driven through the C ABI.

The server side of every round is one ``sf_eval_linear_layer`` job (or one
job inside an ``sf_eval_layers`` batch).  Between rounds a simulated client
decrypts the packed outputs, applies ReLU (order-agnostic, so it works on the
shuffled values), re-encodes at the input scale and encrypts the next round's
input in the order the server's output permutation left it (Sec. 4.3,
Sec. 4.5).  A round may read several earlier activations (the block input of
a residual connection): the client concatenates them, and the round's input
permutation is the concatenation of theirs.

Two client modes.  Fixed point (the default): activations are re-encoded at
the input scale Delta.  Quantised (``act_bits`` set; the paper's integer
setting, Sec. 2 "Quantization" and Sec. 4.5): weights are small integers
encoded at scale 1, activations are unsigned act_bits-bit integers encoded at
Delta, and after ReLU the client requantises every output with the round's
public scale eta, y -> clip(round(y / eta), 0, 2^act_bits - 1), so the
encrypted chain reproduces the quantised cleartext network exactly
(Sec. 6.1's correctness check).

Everything here is host-side orchestration: all arithmetic on ciphertexts
runs in the CUDA library; encryption randomness is drawn by the library from
the seeds given here.
"""
from __future__ import annotations

import time

import numpy as np

import paper_2509_01253_gb300 as sf
from paper_2509_01253_gb300 import protocol
from paper_2509_01253_gb300 import workloads as wl


def _mix(*xs) -> int:
    """SplitMix64-style finaliser over a tuple of ints (seed derivation)."""
    h = 0x243F6A8885A308D3
    for x in xs:
        h = (h ^ (int(x) & 0xFFFFFFFFFFFFFFFF)) * 0x9E3779B97F4A7C15 & 0xFFFFFFFFFFFFFFFF
        h ^= h >> 31
        h = (h * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        h ^= h >> 29
    return h


def requant_scale(spec: wl.RoundSpec) -> int:
    """The round's public requantisation scale eta (Sec. 4.5), a power of
    two: 2^floor(log2(fan_in)), fan_in summed over the round's terms.  With
    weights in {-2..2} and 4-bit inputs an output's spread grows like
    sqrt(fan_in), so this keeps requantised activations inside a few bits."""
    fan = sum(t.kh * t.kw * t.C_in for t in spec.terms)
    return 1 << (fan.bit_length() - 1)


def round_half_away(v: np.ndarray) -> np.ndarray:
    """Round half away from zero (the encoding's rounding rule)."""
    return np.sign(v) * np.floor(np.abs(v) + 0.5)


def requantize(y: np.ndarray, eta: int, act_bits: int) -> np.ndarray:
    """y -> clip(round(y / eta), 0, 2^act_bits - 1) on ReLU outputs (Sec. 4.5)."""
    return np.clip(round_half_away(np.asarray(y, dtype=np.float64) / eta), 0, (1 << act_bits) - 1)


class EncodedNetwork:
    """The rounds of one network with their quantised weights resident on a context.

    act_bits None: fixed point (weights at scale Delta, outputs at Delta^2).
    act_bits set: quantised mode (integer weights at scale 1, outputs at
    Delta, requantisation scale eta per round)."""

    def __init__(self, params, ctx, ps: wl.ParamSet, rounds: list, integer: bool = False, act_bits: int = None,
                 gamma=0):
        self.params, self.ctx, self.ps, self.rounds = params, ctx, ps, rounds
        self.n = 1 << ps.log_n
        self.act_bits = act_bits
        # partial trace extraction level (Sec. 4.3, 4.4), one for all rounds or
        # one per round: at gamma = 2 the client also sends RLWE(m_j(X^3)) for
        # that round and its packed values carry the factor 2
        self.gammas = list(gamma) if isinstance(gamma, (list, tuple)) else [gamma] * len(rounds)
        assert len(self.gammas) == len(rounds) and all(g in (0, 2) for g in self.gammas)
        self.quant = act_bits is not None
        wscale = 1.0 if self.quant else ps.delta
        self.out_scale = ps.delta * wscale
        self.etas = [requant_scale(spec) for spec in rounds] if self.quant else None
        self.layers, self.infos, self.weights = [], [], []
        for spec in rounds:
            ws = wl.round_weights(spec, integer or self.quant)
            W = np.concatenate([w.ravel() for w in ws])
            lay = sf.sf_encode_weights(ctx, spec.terms, W, None, wscale, self.out_scale)
            self.layers.append(lay)
            self.infos.append(sf.sf_layer_get_info(ctx, lay))
            self.weights.append(ws)

    def destroy(self):
        for lay in self.layers:
            sf.sf_layer_destroy(lay)
        self.layers = []

    def max_cts(self) -> int:
        """Largest input + output ciphertext count over the rounds."""
        return max(i["k_in"] + i["n_groups"] for i in self.infos)

    def ks_count(self, r: int, gamma: int = None) -> int:
        """Key switches of round r at extraction level gamma (the round's own
        by default); at gamma = 2 each group of n values saves the n/2 merges
        of the tau_3 level (one trace step when n = 1)."""
        i = self.infos[r]
        g = self.gammas[r] if gamma is None else gamma
        if g != 2:
            return i["ks_count"]
        return i["ks_count"] - i["n_groups"] * (i["group_size"] // 2 if i["group_size"] >= 2 else 1)

    def total_ks(self) -> int:
        """Key switches of all rounds at their extraction levels."""
        return sum(self.ks_count(r) for r in range(len(self.rounds)))


class ClientState:
    """One request's client: its plaintext activations (in the order the
    server's permutation left them) and its session seed.

    acts[name] = (values, perm): values[p] is the activation of original
    index perm[p] (perm None = identity order)."""

    def __init__(self, net: EncodedNetwork, x: np.ndarray, session_seed: int, request_seed: int):
        self.net = net
        self.session_seed = session_seed
        self.request_seed = request_seed
        x = np.asarray(x, dtype=np.float64)
        if net.quant:
            # the image in [0, 1] quantised to act_bits-bit integers
            x = np.clip(round_half_away(x * ((1 << net.act_bits) - 1)), 0, (1 << net.act_bits) - 1)
        self.acts = {"x": (x, None)}
        self.round = 0
        self.trace = []          # per round: (input values in original order, decoded outputs in original order)

    @property
    def done(self) -> bool:
        return self.round >= len(self.net.rounds)

    def sigma_out(self, r: int):
        """Output permutation of round r: a fresh one per round from the session
        seed, none for the last round (its outputs go to the client in order)."""
        if r == len(self.net.rounds) - 1:
            return None
        E = self.net.infos[r]["E_out"]
        return sf.sf_permutation(self.session_seed, r + 1, E)

    def round_input(self, r: int):
        """(stream values, sigma_prev or None) of round r's input."""
        spec = self.net.rounds[r]
        vals, perms, off, any_perm = [], [], 0, False
        for name in spec.inputs:
            v, p = self.acts[name]
            vals.append(v)
            perms.append((np.arange(len(v), dtype=np.int64) if p is None else p.astype(np.int64)) + off)
            any_perm |= p is not None
            off += len(v)
        stream = np.concatenate(vals)
        sigma = np.concatenate(perms).astype(np.uint32) if any_perm else None
        return stream, sigma

    def original_order(self, stream: np.ndarray, sigma) -> np.ndarray:
        if sigma is None:
            return stream.copy()
        out = np.empty_like(stream)
        out[sigma.astype(np.int64)] = stream
        return out

    def encode(self, r: int):
        """Quantised message (int64, stream order) and sigma_prev of round r
        (integer activations times Delta, exactly, in quantised mode)."""
        stream, sigma = self.round_input(r)
        if self.net.quant:
            return stream.astype(np.int64) * int(self.net.ps.delta), sigma, stream
        return sf.sf_encode_input(stream, self.net.ps.delta), sigma, stream

    def encrypt_seed(self, r: int) -> int:
        return _mix(self.request_seed, r, 0xE)

    def power_seed(self, r: int) -> int:
        """Encryption seed of round r's powers (gamma = 2)."""
        return _mix(self.request_seed, r, 0x3)

    def absorb(self, r: int, values: np.ndarray, sigma_out, stream_in=None, sigma_in=None):
        """Store round r's decoded outputs (slot order) as the activation it names."""
        spec = self.net.rounds[r]
        if stream_in is not None:
            y_orig = self.original_order(values, sigma_out)
            self.trace.append((self.original_order(stream_in, sigma_in), y_orig))
        if self.net.quant:
            y = round_half_away(values)             # outputs are integers at scale Delta
            v = requantize(np.maximum(y, 0.0), self.net.etas[r], self.net.act_bits) if spec.relu else y
        else:
            v = np.maximum(values, 0.0) if spec.relu else values.copy()
        self.acts[spec.out] = (v, sigma_out)
        self.round = r + 1

    def logits(self) -> np.ndarray:
        v, p = self.acts[self.net.rounds[-1].out]
        return self.original_order(v, p)


def round_float_reference(net: EncodedNetwork, r: int, x_orig: np.ndarray) -> np.ndarray:
    """f(x) = sum of the round's convolutions in float64 on the given input
    (original order), output in original order."""
    spec = net.rounds[r]
    case = wl.LayerCase(spec.name, spec.terms, net.weights[r], None, x_orig, None, None)
    return wl.float_reference(case)


# ------------------------------------------------------------- one request --

def decode_outputs(net: EncodedNetwork, r: int, residues: np.ndarray) -> np.ndarray:
    info = net.infos[r]
    return sf.sf_decode(net.params, residues, info["n_groups"], net.n // info["group_size"],
                        info["E_out"], net.out_scale * (2 if net.gammas[r] == 2 else 1))


def run_request(net: EncodedNetwork, sk, rk, client: ClientState, stream=None, device: str = "cuda:0",
                keep_trace: bool = False, log: protocol.CommLog = None, session: protocol.ServerSession = None,
                io: list = None, split: list = None):
    """All rounds of one request, one sf_eval_linear_layer call per round.
    Each upload goes through the server's session checks (its session id is
    the client's session seed); `log`, when given, receives every round's
    bytes, server (device) time and client time (encode, encrypt, decrypt,
    decode, activation).  `split`, when given, receives per round the
    (leaf milliseconds, all kernels' milliseconds) of the library's kernel
    timing, which is on for the request (launches bracketed by events, no
    graph replay).  Returns per-round device milliseconds."""
    import torch
    L, n = net.ps.n_data, net.n
    st = stream if stream is not None else torch.cuda.current_stream()
    session = session or protocol.ServerSession(client.session_seed, len(net.rounds))
    ms = []
    timing = sf.sf_ctx_get_option(net.ctx, "kernel_timing")
    if split is not None:
        sf.sf_ctx_set_option(net.ctx, "kernel_timing", 1)
    try:
        _run_rounds(net, sk, rk, client, stream, st, device, keep_trace, log, session, io, split, ms, L, n)
    finally:
        sf.sf_ctx_set_option(net.ctx, "kernel_timing", timing)
    return ms


def _run_rounds(net, sk, rk, client, stream, st, device, keep_trace, log, session, io, split, ms, L, n):
    import torch
    for r in range(len(net.rounds)):
        info = net.infos[r]
        t0 = time.perf_counter()
        msg, sigma_prev, stream_in = client.encode(r)
        d_in = torch.empty((info["k_in"], 2, L, n), dtype=torch.int64, device=device)
        sf.sf_encrypt(net.ctx, sk, msg, client.encrypt_seed(r), d_in, info["k_in"], stream)
        d_pow = None
        if net.gammas[r] == 2:
            d_pow = torch.empty_like(d_in)
            sf.sf_encrypt(net.ctx, sk, sf.sf_client_power(net.params, msg, info["k_in"], 3),
                          client.power_seed(r), d_pow, info["k_in"], stream)
        st.synchronize()
        t_client = time.perf_counter() - t0
        so = client.sigma_out(r)

        def evaluate(rr, payload):
            d_out = torch.empty((info["n_groups"], 2, L, n), dtype=torch.int64, device=device)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if split is not None:
                sf.sf_kernel_stats_reset(net.ctx)
            e0.record(st)
            sf.sf_eval_linear_layer_gamma(net.ctx, net.layers[rr], rk, net.gammas[rr], payload, d_pow, info["k_in"],
                                          sigma_prev, so, d_out, info["n_groups"], st)
            e1.record(st)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            if split is not None:
                stats = sf.sf_kernel_stats(net.ctx)
                split.append((sum(t for name, _, t in stats if name.startswith("leaf")), sum(t for _, _, t in stats)))
            return d_out

        d_out = session.submit(client.session_seed, r, d_in, evaluate)
        if io is not None:
            # (uploaded ciphertexts, packed results, sigma_prev, sigma_out) of the round, for parity checks
            io.append((d_in.cpu().numpy().view(np.uint64), d_out.cpu().numpy().view(np.uint64), sigma_prev, so))
        t0 = time.perf_counter()
        res = np.zeros((info["n_groups"], L, n), dtype=np.uint64)
        sf.sf_decrypt(net.ctx, sk, d_out, info["n_groups"], res, st)
        vals = decode_outputs(net, r, res)
        client.absorb(r, vals, so, stream_in if keep_trace else None, sigma_prev)
        t_client += time.perf_counter() - t0
        if log is not None:
            up, down = protocol.round_bytes(info, L, n, net.gammas[r])
            log.add(r, up, down, ms[-1] / 1e3, t_client)
    return ms


def plan_gammas(net: EncodedNetwork, split: list, margin: float = 0.02, leaf_factor: float = 2.2) -> list:
    """Per-round extraction level from the kernel split of one gamma = 0
    request (run_request's `split`).  Partial extraction (Sec. 4.3, 4.4)
    trades work: at gamma = 2 the server multiplies each round's weights into
    the ciphertexts and into the client's powers, so the leaf kernels' time
    grows by leaf_factor, while the rest of the round, the key switches of
    the packing tree and the trace, shrinks with their count.  The predicted
    gamma = 2 time of round r is leaf_factor leaf_r + (total_r - leaf_r)
    ks_2 / ks_0, and the round takes gamma = 2 when that is below
    (1 - margin) total_r.  The leaves alone would double; the default 2.2
    also carries the powers' input transforms and the plain bottom-level
    merges that the gamma = 2 rounds add (fitted on GB300 over the ResNet-34
    rounds: 2.11 to 2.24).  Early, wide layers keep gamma = 0; the late
    rounds, where key switches dominate, take gamma = 2.  The choice is the
    server's alone: the client sends the powers for exactly the rounds that
    take gamma = 2."""
    assert len(split) == len(net.rounds)
    plan = []
    for r, (leaf, total) in enumerate(split):
        ks0, ks2 = net.ks_count(r, 0), net.ks_count(r, 2)
        pred2 = leaf_factor * leaf + (total - leaf) * (ks2 / ks0 if ks0 else 1.0)
        plan.append(2 if pred2 < (1 - margin) * total else 0)
    return plan


def quant_forward(net: EncodedNetwork, x: np.ndarray, trace: list = None) -> np.ndarray:
    """The quantised cleartext network (Sec. 6.1's reference): the image
    quantised to act_bits bits, each round's integer convolution computed
    exactly, then ReLU and requantisation by the round's eta; returns the
    integer logits.  `trace` receives (input, output) per round, original order."""
    top = (1 << net.act_bits) - 1
    acts = {"x": np.clip(round_half_away(np.asarray(x, dtype=np.float64) * top), 0, top)}
    for r, spec in enumerate(net.rounds):
        inp = np.concatenate([acts[name] for name in spec.inputs])
        y = round_float_reference(net, r, inp)      # integers below 2^53: exact in float64
        if trace is not None:
            trace.append((inp, y))
        acts[spec.out] = requantize(np.maximum(y, 0.0), net.etas[r], net.act_bits) if spec.relu else y
    return acts[net.rounds[-1].out]


def float_forward(net: EncodedNetwork, x: np.ndarray, trace: list = None) -> np.ndarray:
    """The plaintext network in float64 with the same weights: rounds in
    order, ReLU where the round applies it; returns the logits."""
    acts = {"x": np.asarray(x, dtype=np.float64)}
    for r, spec in enumerate(net.rounds):
        inp = np.concatenate([acts[name] for name in spec.inputs])
        y = round_float_reference(net, r, inp)
        if trace is not None:
            trace.append((inp, y))
        acts[spec.out] = np.maximum(y, 0.0) if spec.relu else y
    return acts[net.rounds[-1].out]
