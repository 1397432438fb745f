"""Protocol bookkeeping (host logic, no GPU): session and round checks,
resending the last packed result after a lost download, resuming after a
reconnect, communication volume and end-to-end latency at a bandwidth.  The
last test runs a client and a server as two gloo ranks that exchange real
messages, with one reply dropped on the wire."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp

from paper_2509_01253_gb300 import protocol as P
from paper_2509_01253_gb300 import workloads as wl


class _Counter:
    def __init__(self):
        self.calls = []

    def __call__(self, r, payload):
        self.calls.append(r)
        return ("packed", r, payload)


def test_rounds_in_order_are_evaluated_once():
    s, ev = P.ServerSession(77, 3), _Counter()
    for r in range(3):
        assert s.submit(77, r, f"ct{r}", ev) == ("packed", r, f"ct{r}")
    assert ev.calls == [0, 1, 2] and s.finished and s.evaluations == 3 and s.resends == 0


def test_refused_messages():
    s, ev = P.ServerSession(5, 4), _Counter()
    with pytest.raises(P.ProtocolError) as e:
        s.submit(6, 0, "x", ev)                  # another session
    assert e.value.code == "session"
    with pytest.raises(P.ProtocolError) as e:
        s.submit(5, 1, "x", ev)                  # skips round 0
    assert e.value.code == "order"
    s.submit(5, 0, "x", ev)
    s.submit(5, 1, "x", ev)
    with pytest.raises(P.ProtocolError) as e:
        s.submit(5, 0, "x", ev)                  # two rounds back: not a resend
    assert e.value.code == "order"
    s.submit(5, 2, "x", ev)
    s.submit(5, 3, "x", ev)
    assert s.submit(5, 3, "again", ev) == ("packed", 3, "x")   # a resend after the last round
    with pytest.raises(P.ProtocolError) as e:
        s.submit(5, 4, "x", ev)                  # past the last round
    assert e.value.code == "done"
    with pytest.raises(P.ProtocolError):
        s.complete(2, None)                      # completing a round that is not in progress
    assert ev.calls == [0, 1, 2, 3]
    with pytest.raises(ValueError):
        P.ServerSession(1, 0)


def test_resend_returns_the_kept_result_without_evaluating():
    s, ev = P.ServerSession(9, 5), _Counter()
    first = s.submit(9, 0, "ct0", ev)
    again = s.submit(9, 0, "ct0 resent", ev)     # the client lost the download
    assert again is first and ev.calls == [0] and s.resends == 1
    assert s.submit(9, 1, "ct1", ev) == ("packed", 1, "ct1")


def test_resume_after_a_disconnect():
    s, ev = P.ServerSession(3, 4), _Counter()
    s.submit(3, 0, "a", ev)
    s.submit(3, 1, "b", ev)                      # the connection drops before the client reads this
    nxt, last = s.resume(3)
    assert nxt == 2 and last == ("packed", 1, "b")
    with pytest.raises(P.ProtocolError):
        s.resume(4)
    assert P.ServerSession(8, 2).resume(8) == (0, None)   # nothing evaluated yet


def test_round_shapes_and_bytes():
    # the conv16 benchmark round: one input ciphertext, two packed groups of 8192
    sh = P.round_shape(16384, 16384, 1 << 14)
    assert sh == {"k_in": 1, "group_size": 8192, "n_groups": 2}
    assert P.round_bytes(sh, 3, 1 << 14) == (786_432, 1_572_864)
    # the 64x64 FC round at N = 2^12: 64 outputs in one group of 64
    assert P.round_shape(64, 64, 1 << 12) == {"k_in": 1, "group_size": 64, "n_groups": 1}
    # ragged last group, several input ciphertexts
    assert P.round_shape(3 * 4096 + 1, 5000, 4096) == {"k_in": 4, "group_size": 2048, "n_groups": 3}
    # ResNet-20 at N = 2^14, 3 data limbs: 24 input ciphertexts up (stage 0's second convs read the block
    # input and the shortcut, 2 each, as does the strided s1b0c2 over 16384 + 8192 values; every other round
    # reads one) and 27 packed ciphertexts down (the seven 16384-output rounds of stage 0 and the stem
    # fill two groups of 8192, the other 13 rounds one group): 18.9 MB up, 21.2 MB down per request
    N = 1 << 14
    shapes = [P.round_shape(wl.round_input_size(r), wl.round_output_size(r), N) for r in wl.resnet_rounds("resnet20")]
    assert sum(s["k_in"] for s in shapes) == 24 and sum(s["n_groups"] for s in shapes) == 27
    ct = P.ciphertext_bytes(3, N)
    assert ct == 786_432 and 24 * ct == 18_874_368 and 27 * ct == 21_233_664


def test_e2e_latency_model():
    log = P.CommLog()
    log.add(0, 1_000_000, 2_000_000, server_s=1.5, client_s=0.25)
    log.add(1, 500_000, 500_000, server_s=0.5, client_s=0.25)
    assert (log.up_bytes, log.down_bytes) == (1_500_000, 2_500_000)
    assert log.e2e_seconds(1.25e6) == pytest.approx(2.0 + 0.5 + 4_000_000 / 1.25e6)
    summ = log.summary((1.25, 100.0))
    assert summ["e2e_s_at_MBps"]["100.0"] == pytest.approx(2.5 + 0.04)
    with pytest.raises(ValueError):
        log.e2e_seconds(0)


# ------------------------------------------------ client and server ranks --

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _peer(rank, port, n_rounds, drop_round, out):
    """Rank 0 serves, rank 1 is the client.  A message is a tensor
    [session, round, value]; the server's reply for `drop_round` is lost on
    the wire the first time (it sends a marker the client treats as a
    timeout), and the client uploads that round again."""
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    session_id = 4242
    if rank == 0:
        srv, calls = P.ServerSession(session_id, n_rounds), []
        dropped = False

        def evaluate(r, value):
            calls.append(r)
            return value * 2 + r                 # stands in for the packed result

        while not srv.finished or not dropped:
            msg = torch.zeros(3, dtype=torch.int64)
            dist.recv(msg, src=1)
            sid, r, v = (int(x) for x in msg)
            try:
                res = srv.submit(sid, r, v, evaluate)
                reply = torch.tensor([sid, r, res], dtype=torch.int64)
            except P.ProtocolError:
                reply = torch.tensor([sid, -2, 0], dtype=torch.int64)
            if r == drop_round and not dropped:
                dropped = True
                reply = torch.tensor([sid, -1, 0], dtype=torch.int64)   # lost on the wire
            dist.send(reply, dst=1)
            if srv.finished and dropped:
                break
        out["calls"], out["resends"] = calls, srv.resends
    else:
        results, r, value, refused = [], 0, 1, 0
        # one message the server must refuse: a round ahead of the session
        dist.send(torch.tensor([session_id, 5, 0], dtype=torch.int64), dst=0)
        reply = torch.zeros(3, dtype=torch.int64)
        dist.recv(reply, src=0)
        refused += int(reply[1]) == -2
        while r < n_rounds:
            dist.send(torch.tensor([session_id, r, value], dtype=torch.int64), dst=0)
            reply = torch.zeros(3, dtype=torch.int64)
            dist.recv(reply, src=0)
            if int(reply[1]) == -1:              # no answer: send the same round again
                continue
            results.append(int(reply[2]))
            value = int(reply[2]) % 1000         # the next round's input depends on this one's output
            r += 1
        out["results"], out["refused"] = results, refused
    dist.barrier()
    dist.destroy_process_group()


def test_client_and_server_ranks_with_a_lost_reply():
    port, n_rounds, drop_round = _free_port(), 4, 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_peer, args=(port, n_rounds, drop_round, out), nprocs=2, join=True)
        res = dict(out)
    # every round evaluated exactly once although round 2 was uploaded twice
    assert res["calls"] == [0, 1, 2, 3] and res["resends"] == 1 and res["refused"] == 1
    want, v = [], 1
    for r in range(n_rounds):
        y = v * 2 + r
        want.append(y)
        v = y % 1000
    assert res["results"] == want


@pytest.mark.parametrize("kind,pset", [("resnet20", "conv16"), ("resnet18", "r18"), ("resnet34", "r34")])
def test_round_shapes_agree_with_the_oracle(oracle, kind, pset):
    """The protocol's round shapes (what it counts as bytes) against the
    oracle's own packing rule, round by round: group size, packed ciphertexts
    and the key switches those groups cost."""
    ps = wl.PARAMS[pset]
    N = 1 << ps.log_n
    prm = oracle.Params(ps.log_n, N, ps.n_data, ps.n_special, [], [])
    for spec in wl.resnet_rounds(kind):
        e_in, e_out = wl.round_input_size(spec), wl.round_output_size(spec)
        sh = P.round_shape(e_in, e_out, N)
        n = oracle.group_size(prm, e_out)
        assert sh["group_size"] == n, spec.name
        assert sh["n_groups"] * n >= e_out > (sh["n_groups"] - 1) * n, spec.name
        assert sh["k_in"] * N >= e_in > (sh["k_in"] - 1) * N, spec.name
        log_n_over_n = ps.log_n - (n.bit_length() - 1)
        assert oracle.ks_count(prm, e_out) == sh["n_groups"] * ((n - 1) + log_n_over_n), spec.name
