"""Multi-round encrypted inference and the continuous-batching server on the
GPU: a small ResNet-shaped network end to end against its float64 forward
pass, and every request's result identical alone and inside a served mix of
networks, parameter sets and client keys."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2509_01253_gb300 as sf  # noqa: E402
from paper_2509_01253_gb300 import network as nw  # noqa: E402
from paper_2509_01253_gb300 import protocol  # noqa: E402
from paper_2509_01253_gb300 import serve  # noqa: E402
from paper_2509_01253_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module")
def pools():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    p = {"p12": serve.Pool(wl.PARAMS["fc64"], ["tiny_a"], 2, 0, key_seed=11),
         "p14": serve.Pool(wl.PARAMS["conv16"], ["tiny_a", "tiny_b", "resnet20"], 2, 0, key_seed=21,
                           engine_budget=1 << 30)}
    yield p
    for x in p.values():
        x.destroy()


def _alone(pool, net, key, seed, log=None, session=None):
    req = serve.make_request(0, net, key, seed)
    client = nw.ClientState(pool.nets[net], req.x, req.session_seed, req.request_seed)
    nw.run_request(pool.nets[net], pool.sks[key], pool.rks[key], client, keep_trace=True, log=log, session=session)
    return client


def test_request_protocol_accounting(pools):
    """One request through the session checks: every round evaluated once,
    the communication log equal to the rounds' ciphertext counts, and the
    host-side round shapes equal to the library's layer info."""
    pool, net = pools["p14"], "tiny_b"
    encnet = pool.nets[net]
    req = serve.make_request(0, net, 0, 51)
    session = protocol.ServerSession(req.session_seed, len(encnet.rounds))
    log = protocol.CommLog()
    _alone(pool, net, 0, 51, log=log, session=session)
    assert session.finished and session.evaluations == len(encnet.rounds) and session.resends == 0
    ct = protocol.ciphertext_bytes(pool.L, pool.n)
    assert log.up_bytes == sum(i["k_in"] for i in encnet.infos) * ct
    assert log.down_bytes == sum(i["n_groups"] for i in encnet.infos) * ct
    assert all(x.server_s > 0 and x.client_s > 0 for x in log.rounds)
    for spec, info in zip(encnet.rounds, encnet.infos):
        sh = protocol.round_shape(wl.round_input_size(spec), wl.round_output_size(spec), pool.n)
        assert (sh["k_in"], sh["group_size"], sh["n_groups"]) == (info["k_in"], info["group_size"], info["n_groups"])
    # a resend of the last round is answered from the kept result
    last = len(encnet.rounds) - 1
    assert session.submit(req.session_seed, last, None, lambda r, p: pytest.fail("evaluated again")) is \
        session.last_result


@pytest.mark.parametrize("pool_name,net", [("p12", "tiny_a"), ("p14", "tiny_b")])
def test_network_rounds_match_float64(pools, pool_name, net):
    pool = pools[pool_name]
    client = _alone(pool, net, 1, 5)
    encnet = pool.nets[net]
    assert len(client.trace) == len(encnet.rounds)
    # every round against the plaintext layer on the client's actual input
    for r, (x_in, y) in enumerate(client.trace):
        ref = nw.round_float_reference(encnet, r, x_in)
        assert np.abs(y - ref).max() <= 1e-3, (net, r)
    # and the whole chain against the float64 network
    ref = nw.float_forward(encnet, wl.network_input(net, 5))
    assert np.abs(client.logits() - ref).max() <= 1e-3


def test_served_results_equal_alone(pools):
    route = {"tiny_a": "p12", "tiny_b": "p14"}
    specs = [("tiny_a", 0, 31), ("tiny_b", 1, 32), ("tiny_a", 1, 33), ("tiny_b", 0, 34), ("tiny_b", 1, 35),
             ("tiny_a", 0, 36), ("tiny_b", 0, 37)]
    alone = {seed: _alone(pools[route[net]], net, key, seed).logits() for net, key, seed in specs}
    srv = serve.Server(pools, route, mem_budget=1 << 34, max_queue=16, max_active=3, max_batch=2)
    srv.start()
    import time
    for i, (net, key, seed) in enumerate(specs):
        assert srv.submit(serve.make_request(i, net, key, seed))
        if i == 3:
            time.sleep(0.05)        # the rest arrive while the first are on the device
    t_end = time.perf_counter() + 300
    while not srv.idle() and time.perf_counter() < t_end and not srv.errors:
        time.sleep(0.01)
    srv.shutdown()
    assert len(srv.completed) == len(specs)
    assert max(b[1] for b in srv.batches) == 2        # calls held several requests
    for req in srv.completed:                         # the server's session of every request ran to the end
        assert req.session.finished and req.session.evaluations == len(pools[route[req.net]].nets[req.net].rounds)
        assert req.up_bytes > 0 and req.down_bytes > 0
    for req in srv.completed:
        assert np.array_equal(req.logits, alone[req.request_seed]), req.request_seed


def test_served_resnet20_mix_equals_alone(pools):
    """Full ResNet-20 requests (N = 2^14, groups of 8192 split into units of
    leaves under a 1 GiB engine budget) under two client keys, three at a time
    in one engine call: identical to each request alone."""
    route = {"resnet20": "p14"}
    specs = [("resnet20", 0, 41), ("resnet20", 1, 42), ("resnet20", 0, 43)]
    alone = {seed: _alone(pools["p14"], net, key, seed).logits() for net, key, seed in specs}
    srv = serve.Server({"p14": pools["p14"]}, route, mem_budget=1 << 36, max_queue=8, max_active=3, max_batch=3)
    srv.start()
    import time
    for i, (net, key, seed) in enumerate(specs):
        assert srv.submit(serve.make_request(i, net, key, seed))
    t_end = time.perf_counter() + 600
    while not srv.idle() and time.perf_counter() < t_end and not srv.errors:
        time.sleep(0.02)
    srv.shutdown()
    assert len(srv.completed) == 3
    assert max(b[1] for b in srv.batches) == 3
    for req in srv.completed:
        assert np.array_equal(req.logits, alone[req.request_seed]), req.request_seed
    ref = nw.float_forward(pools["p14"].nets["resnet20"], wl.network_input("resnet20", 41))
    assert np.abs(alone[41] - ref).max() <= 1e-3


@pytest.mark.gpu
def test_quantised_request_matches_oracle_rounds_and_cleartext(oracle):
    """Integer mode over a whole request (tiny_a at N = 2^12, 2 x 30-bit + 1,
    4-bit activations, integer weights at scale 1, Delta = 2^25): every round's
    packed residues equal the oracle's round on the same uploaded ciphertexts
    (extraction, unshuffle, linear step, shuffle, packing), every round's
    decrypted outputs equal the quantised cleartext round exactly, and so do
    the final logits (Sec. 6.1's check), with the client requantising by each
    round's eta between rounds (Sec. 4.5)."""
    import paper_2509_01253_gb300 as sf
    from _gpu import Session, oracle_params
    ps = wl.PARAMS["fc64"]
    s = Session.from_set(ps, sk_seed=91, rk_seed=92)
    net = None
    try:
        net = nw.EncodedNetwork(s.params, s.ctx, ps, wl.resnet_rounds("tiny_a"), act_bits=4)
        x = wl.network_input("tiny_a", 93)
        client = nw.ClientState(net, x, session_seed=94, request_seed=95)
        io = []
        nw.run_request(net, s.sk, s.rk, client, keep_trace=True, io=io)
        trace = []
        logits = nw.quant_forward(net, x, trace)
        assert np.array_equal(client.logits(), logits)
        prm = oracle_params(oracle, ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits)
        s_o = oracle.keygen(prm, 91)
        keys = oracle.rotation_keys(prm, s_o, 92)
        for r, (spec, (cts, out, sp, so)) in enumerate(zip(net.rounds, io)):
            x_in, y = client.trace[r]
            assert np.array_equal(x_in, trace[r][0]) and np.array_equal(np.floor(y + 0.5), trace[r][1]), spec.name
            terms = [oracle.ConvTerm(t.in_offset, t.H, t.W, t.C_in, t.C_out, t.kh, t.kw, t.stride, t.pad)
                     for t in spec.terms]
            lay = oracle.make_layer(terms, net.weights[r], None, 1.0, ps.delta)
            want = oracle.eval_linear_layer(prm, lay, keys, cts, sp, so)
            assert (out == want).all(), spec.name
    finally:
        if net is not None:
            net.destroy()
        s.close()


@pytest.fixture(scope="module")
def pool_g2():
    """A gamma = 2 pool at N = 2^14 with the keys of the p14 pool (same key seed)."""
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    p = serve.Pool(wl.PARAMS["conv16"], ["tiny_b", "resnet20"], 2, 0, key_seed=21, engine_budget=1 << 30, gamma=2)
    yield p
    p.destroy()


@pytest.mark.gpu
def test_gamma2_request_matches_float64(pools, pool_g2):
    """A whole request with partial trace extraction at gamma = 2 (the client
    sends RLWE(m(X^3)) beside every input ciphertext, every round skips the
    tau_3 level): each round within 1e-3 of float64 on its actual input, the
    logits within 1e-3 of the float64 network and of the gamma = 0 request, and
    the upload doubled."""
    log2, log0 = protocol.CommLog(), protocol.CommLog()
    c2 = _alone(pool_g2, "tiny_b", 1, 5, log=log2)
    c0 = _alone(pools["p14"], "tiny_b", 1, 5, log=log0)
    encnet = pool_g2.nets["tiny_b"]
    for r, (x_in, y) in enumerate(c2.trace):
        assert np.abs(y - nw.round_float_reference(encnet, r, x_in)).max() <= 1e-3, r
    ref = nw.float_forward(encnet, wl.network_input("tiny_b", 5))
    assert np.abs(c2.logits() - ref).max() <= 1e-3
    assert np.abs(c2.logits() - c0.logits()).max() <= 1e-3
    assert log2.up_bytes == 2 * log0.up_bytes and log2.down_bytes == log0.down_bytes


@pytest.mark.gpu
def test_served_gamma2_mix_equals_alone(pool_g2):
    """ResNet-20 and tiny_b requests at gamma = 2 under two client keys, three
    at a time in one engine call (sf_eval_layers_gamma): identical to each
    request alone."""
    route = {"resnet20": "g2", "tiny_b": "g2"}
    specs = [("resnet20", 0, 61), ("tiny_b", 1, 62), ("resnet20", 1, 63)]
    alone = {seed: _alone(pool_g2, net, key, seed).logits() for net, key, seed in specs}
    srv = serve.Server({"g2": pool_g2}, route, mem_budget=1 << 36, max_queue=8, max_active=3, max_batch=3)
    srv.start()
    import time
    for i, (net, key, seed) in enumerate(specs):
        assert srv.submit(serve.make_request(i, net, key, seed))
    t_end = time.perf_counter() + 600
    while not srv.idle() and time.perf_counter() < t_end and not srv.errors:
        time.sleep(0.02)
    srv.shutdown()
    assert not srv.errors and len(srv.completed) == 3
    for req in srv.completed:
        assert np.array_equal(req.logits, alone[req.request_seed]), req.request_seed
    ref = nw.float_forward(pool_g2.nets["resnet20"], wl.network_input("resnet20", 61))
    assert np.abs(alone[61] - ref).max() <= 1e-3


@pytest.mark.gpu
def test_per_round_gamma_plan_request_and_served(pools, pool_g2):
    """Extraction level per round: the planner turns the kernel split of a
    gamma = 0 request into one level per round; a request whose rounds
    alternate gamma = 0 and 2 (the client sends powers only for the latter)
    is within 1e-3 of float64 and of the gamma = 0 request, uploads the
    powers of exactly those rounds, and gives identical logits when served
    two at a time (sf_eval_layers_gamma with and without powers in one call)."""
    p0 = pools["p14"]
    net0 = p0.nets["tiny_b"]
    split = []
    req = serve.make_request(0, "tiny_b", 0, 71)
    client = nw.ClientState(net0, req.x, req.session_seed, req.request_seed)
    nw.run_request(net0, p0.sks[0], p0.rks[0], client, split=split)
    assert sf.sf_ctx_get_option(p0.ctx, "kernel_timing") == 0
    assert len(split) == len(net0.rounds) and all(0 < leaf <= tot for leaf, tot in split)
    plan = nw.plan_gammas(net0, split)
    assert len(plan) == len(net0.rounds) and set(plan) <= {0, 2}
    # a round whose time is all key switches takes gamma = 2, one all leaves keeps 0
    assert nw.plan_gammas(net0, [(0.0, 1.0)] * len(net0.rounds)) == [2] * len(net0.rounds)
    assert nw.plan_gammas(net0, [(1.0, 1.0)] * len(net0.rounds)) == [0] * len(net0.rounds)
    net = pool_g2.nets["tiny_b"]
    saved = list(net.gammas)
    try:
        net.gammas = [2 if r % 2 else 0 for r in range(len(net.rounds))]
        log_m, log_0 = protocol.CommLog(), protocol.CommLog()
        cm = _alone(pool_g2, "tiny_b", 1, 72, log=log_m)
        c0 = _alone(pools["p14"], "tiny_b", 1, 72, log=log_0)
        for r, (x_in, y) in enumerate(cm.trace):
            assert np.abs(y - nw.round_float_reference(net, r, x_in)).max() <= 1e-3, r
        assert np.abs(cm.logits() - c0.logits()).max() <= 1e-3
        ct = protocol.ciphertext_bytes(pool_g2.L, pool_g2.n)
        extra = sum(i["k_in"] for i, g in zip(net.infos, net.gammas) if g == 2) * ct
        assert log_m.up_bytes == log_0.up_bytes + extra and log_m.down_bytes == log_0.down_bytes
        assert net.total_ks() == sum(net.ks_count(r, g) for r, g in enumerate(net.gammas))
        srv = serve.Server({"g2": pool_g2}, {"tiny_b": "g2"}, mem_budget=1 << 36, max_queue=4, max_active=2,
                           max_batch=2)
        srv.start()
        import time
        for i, seed in enumerate((72, 73)):
            assert srv.submit(serve.make_request(i, "tiny_b", 1, seed))
        t_end = time.perf_counter() + 300
        while not srv.idle() and time.perf_counter() < t_end and not srv.errors:
            time.sleep(0.02)
        srv.shutdown()
        assert not srv.errors and len(srv.completed) == 2
        alone73 = _alone(pool_g2, "tiny_b", 1, 73).logits()
        for r in srv.completed:
            assert np.array_equal(r.logits, cm.logits() if r.request_seed == 72 else alone73), r.request_seed
    finally:
        net.gammas = saved
