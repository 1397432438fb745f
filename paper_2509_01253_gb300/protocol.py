"""Protocol bookkeeping around the server rounds: session and round checks,
resumption after a lost connection, and communication accounting.

The server side of every round is the linear-layer round of Sec. 4.4; the
client decrypts, applies the activation and re-encrypts between rounds
(Sec. 4.5).  This module holds what the paper's protocol needs around that:

* Every upload names its session and its round (the round number also seeds
  that round's output permutation, Sec. 4.4 "Shuffle").  The server
  evaluates round r of a session only when r is the round it expects next.
  An upload of the round it has just evaluated comes from a client that lost
  the download, or reconnected, and sent again: the server answers with the
  packed result it kept and does not evaluate again.  Any other round, and
  any upload for another session, is refused.
* A client that reconnects asks where to continue (Sec. 4.6, client
  availability: the server keeps the current encrypted state and resumes
  once the client is back): the answer is the next round the server
  expects, with the packed result of the round before it, which the client
  may not have received.
* Communication: round r moves its k_in input ciphertexts up and its
  ceil(E'/n) packed ciphertexts down, 2 L N words of 8 bytes each.  The
  end-to-end latency of a request is its client time plus its server time
  plus all bytes exchanged over a symmetric link of a given bandwidth, the
  model of the paper's metrics (Sec. 6.2) and network study (Sec. 6.3, 0.1
  to 300 MB/s; 1.25 MB/s in its E2E comparison).

Host-side only: no ciphertext arithmetic happens here.
"""
from __future__ import annotations

from dataclasses import dataclass, field

WORD_BYTES = 8
PAPER_BANDWIDTHS_MBPS = (0.1, 0.3, 1.0, 1.25, 3.0, 10.0, 30.0, 100.0, 300.0)


class ProtocolError(RuntimeError):
    """A message the server refuses: `code` is "session" (another session's
    message), "order" (not the next round, nor a resend of the last one) or
    "done" (the session has run all its rounds and nothing to resend)."""

    def __init__(self, code: str, message: str):
        super().__init__(message)
        self.code = code


def ciphertext_bytes(L: int, n: int) -> int:
    """One RLWE ciphertext (a, b) with L limbs of N residues."""
    return 2 * L * n * WORD_BYTES


def round_shape(E_in: int, E_out: int, n: int) -> dict:
    """The ciphertext counts of a round from its sizes, as the library's
    layer info reports them: k_in = ceil(E/N) input ciphertexts (Sec. 4.3),
    packing groups of min(N/2, next power of two >= E') outputs (Sec. 4.4),
    ceil(E'/group) packed ciphertexts."""
    if E_in < 1 or E_out < 1:
        raise ValueError("a round has at least one input and one output")
    group = min(n // 2, 1 << (E_out - 1).bit_length())
    return {"k_in": -(-E_in // n), "group_size": group, "n_groups": -(-E_out // group)}


def round_bytes(info: dict, L: int, n: int, gamma: int = 0) -> tuple:
    """(upload, download) bytes of one round: k_in input ciphertexts up (and
    as many powers RLWE(m_j(X^3)) at gamma = 2, Sec. 4.3), n_groups packed
    ciphertexts down."""
    ct = ciphertext_bytes(L, n)
    return info["k_in"] * ct * (2 if gamma == 2 else 1), info["n_groups"] * ct


class ServerSession:
    """The server's state of one session: the next round it expects and the
    packed result of the last round it evaluated.

    `begin(session_id, r)` checks an upload: True when round r is to be
    evaluated, False when it is a resend of the last round (take the kept
    result from `last_result`).  `complete(r, result)` stores the result of
    round r and advances the session.  `submit` runs both around an
    evaluation callback."""

    def __init__(self, session_id: int, n_rounds: int):
        if n_rounds < 1:
            raise ValueError("a session has at least one round")
        self.session_id = session_id
        self.n_rounds = n_rounds
        self.next_round = 0
        self.last_round = None
        self.last_result = None
        self.evaluations = 0
        self.resends = 0

    @property
    def finished(self) -> bool:
        return self.next_round >= self.n_rounds

    def begin(self, session_id: int, r: int) -> bool:
        if session_id != self.session_id:
            raise ProtocolError("session", f"upload for session {session_id} reached session {self.session_id}")
        if r == self.next_round and not self.finished:
            return True
        if self.last_round is not None and r == self.last_round:
            self.resends += 1
            return False
        if self.finished:
            raise ProtocolError("done", f"session {self.session_id} has run all {self.n_rounds} rounds")
        raise ProtocolError("order", f"round {r} of session {self.session_id}: expected round {self.next_round}")

    def complete(self, r: int, result):
        if r != self.next_round:
            raise ProtocolError("order", f"completing round {r}, but round {self.next_round} is the one in progress")
        self.last_round, self.last_result = r, result
        self.next_round = r + 1
        self.evaluations += 1

    def submit(self, session_id: int, r: int, payload, evaluate):
        """The server's answer to an upload of round r: evaluate(r, payload)
        for the next round, the kept result for a resend of the last one."""
        if not self.begin(session_id, r):
            return self.last_result
        result = evaluate(r, payload)
        self.complete(r, result)
        return result

    def resume(self, session_id: int) -> tuple:
        """A reconnecting client: (next round expected, packed result of the
        round before it or None)."""
        if session_id != self.session_id:
            raise ProtocolError("session", f"resume of session {session_id} reached session {self.session_id}")
        return self.next_round, self.last_result


@dataclass
class RoundRecord:
    r: int
    up_bytes: int
    down_bytes: int
    server_s: float
    client_s: float


@dataclass
class CommLog:
    """Per-round bytes and times of one request."""
    rounds: list = field(default_factory=list)

    def add(self, r: int, up_bytes: int, down_bytes: int, server_s: float, client_s: float):
        self.rounds.append(RoundRecord(r, up_bytes, down_bytes, server_s, client_s))

    @property
    def up_bytes(self) -> int:
        return sum(x.up_bytes for x in self.rounds)

    @property
    def down_bytes(self) -> int:
        return sum(x.down_bytes for x in self.rounds)

    @property
    def server_s(self) -> float:
        return sum(x.server_s for x in self.rounds)

    @property
    def client_s(self) -> float:
        return sum(x.client_s for x in self.rounds)

    def e2e_seconds(self, bandwidth_bytes_per_s: float) -> float:
        """Client time + server time + every byte over a symmetric link."""
        if bandwidth_bytes_per_s <= 0:
            raise ValueError("bandwidth must be positive")
        return self.client_s + self.server_s + (self.up_bytes + self.down_bytes) / bandwidth_bytes_per_s

    def summary(self, bandwidths_mbps=PAPER_BANDWIDTHS_MBPS) -> dict:
        return {"rounds": len(self.rounds), "upload_bytes": self.up_bytes, "download_bytes": self.down_bytes,
                "server_s": self.server_s, "client_s": self.client_s,
                "e2e_s_at_MBps": {str(b): self.e2e_seconds(b * 1e6) for b in bandwidths_mbps}}
