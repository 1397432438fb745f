"""Continuous-batching server for encrypted inference requests.

A request is one client's encrypted inference of one network: every round
is a server linear-layer round (Sec. 4.4) and between rounds the client
decrypts, applies ReLU and re-encrypts (Sec. 4.5; simulated here).  The
server keeps every network's quantised weights and every client's rotation
keys resident on the device and runs one worker per parameter set (one
context, one CUDA stream).  Each worker iteration takes the pending round of
every request it holds -- requests at different depths of different
networks, under different client keys -- and evaluates them together in one
``sf_eval_layers`` call; requests admitted while a call is on the device join
the next iteration.  Workers of different parameter sets run concurrently,
so their launches overlap on the GPU.

Admission: an arriving request waits in a FIFO queue; the head is admitted
when the device memory it may hold (its largest round's input plus output
ciphertexts) fits the budget and its worker holds fewer than `max_active`
requests.  A request that finds the queue full is rejected.

All ciphertext arithmetic runs in the CUDA library; this module schedules.
"""
from __future__ import annotations

import collections
import json
import threading
import time
from dataclasses import dataclass, field

import numpy as np

import paper_2509_01253_gb300 as sf
from paper_2509_01253_gb300 import network as nw
from paper_2509_01253_gb300 import protocol
from paper_2509_01253_gb300 import workloads as wl


@dataclass
class Request:
    rid: int
    net: str
    key: int                 # client key id
    x: np.ndarray            # the client's input image (flattened h, w, c)
    session_seed: int
    request_seed: int
    arrival: float = 0.0
    admitted: float = None
    finished: float = None
    reserve: int = 0
    client: nw.ClientState = None
    logits: np.ndarray = None
    rounds_run: int = 0
    # the server's view of the session: round checks and bytes moved
    session: protocol.ServerSession = None
    up_bytes: int = 0
    down_bytes: int = 0
    # the pending round on the device
    d_in: object = None
    d_pow: object = None     # the client's powers at gamma = 2
    d_out: object = None
    sigma_prev: object = None
    sigma_out: object = None
    round_ms: list = field(default_factory=list)


class Pool:
    """One parameter set: context, stream, resident weights and client keys."""

    def __init__(self, ps: wl.ParamSet, nets: list, n_clients: int, device: int = 0, key_seed: int = 7000,
                 engine_budget: int = 16 << 30, ks_batch: int = None, priority: int = 0, gamma=0):
        import torch
        self.torch = torch
        self.ps = ps
        self.params = sf.sf_params_create(ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits,
                                          ps.sigma)
        self.ctx = sf.sf_ctx_create(self.params, device)
        sf.sf_ctx_set_option(self.ctx, "mem_budget", engine_budget)
        if ks_batch:
            sf.sf_ctx_set_option(self.ctx, "ks_batch", ks_batch)
        self.device = f"cuda:{device}"
        self.sks = [sf.sf_keygen(self.ctx, key_seed + 2 * c) for c in range(n_clients)]
        self.rks = [sf.sf_gen_rotation_keys(self.ctx, sk, None, key_seed + 2 * c + 1) for c, sk in enumerate(self.sks)]
        # partial trace extraction level (Sec. 4.3, 4.4): one for every round of
        # every network, or per network a per-round list (a plan_gammas result)
        self.nets = {name: nw.EncodedNetwork(self.params, self.ctx, ps, wl.resnet_rounds(name),
                                             gamma=gamma[name] if isinstance(gamma, dict) else gamma)
                     for name in nets}
        # CUDA stream priority (lower = higher): the pool of short requests runs
        # above the pool of long ones, so its launches take SMs as they free up
        self.stream = torch.cuda.Stream(device=device, priority=priority)
        self.n, self.L = 1 << ps.log_n, ps.n_data
        self.ct_bytes = 2 * self.L * self.n * 8
        # decoded values beyond this are decryption garbage, not activations
        self.activation_bound = 1e9
        self.last_call = []

    def reserve_of(self, net: str) -> int:
        # input (and, at gamma = 2, the powers) plus output ciphertexts of the largest round
        e = self.nets[net]
        per = max(i["k_in"] * (2 if g == 2 else 1) + i["n_groups"] for i, g in zip(e.infos, e.gammas))
        return per * self.ct_bytes

    def new_client(self, req: Request) -> nw.ClientState:
        req.session = protocol.ServerSession(req.session_seed, len(self.nets[req.net].rounds))
        return nw.ClientState(self.nets[req.net], req.x, req.session_seed, req.request_seed)

    def bind_thread(self):
        self.torch.cuda.set_device(self.stream.device)

    # ---- client side (simulated) and buffers
    def prepare(self, req: Request):
        """Encrypt the request's next round input into fresh device buffers."""
        torch = self.torch
        net = self.nets[req.net]
        r = req.client.round
        info = net.infos[r]
        msg, sp, _ = req.client.encode(r)
        # the upload of round r: checked against the session's next round
        if not req.session.begin(req.session_seed, r):
            raise protocol.ProtocolError("order", f"request {req.rid}: round {r} was evaluated already")
        req.up_bytes += protocol.round_bytes(info, self.L, self.n, net.gammas[r])[0]
        req.d_in = torch.empty((info["k_in"], 2, self.L, self.n), dtype=torch.int64, device=self.device)
        sf.sf_encrypt(self.ctx, self.sks[req.key], msg, req.client.encrypt_seed(r), req.d_in, info["k_in"],
                      self.stream)
        req.d_pow = None
        if net.gammas[r] == 2:
            req.d_pow = torch.empty_like(req.d_in)
            sf.sf_encrypt(self.ctx, self.sks[req.key], sf.sf_client_power(self.params, msg, info["k_in"], 3),
                          req.client.power_seed(r), req.d_pow, info["k_in"], self.stream)
        req.d_out = torch.empty((info["n_groups"], 2, self.L, self.n), dtype=torch.int64, device=self.device)
        req.sigma_prev = sp
        req.sigma_out = req.client.sigma_out(r)

    def absorb(self, req: Request):
        """Decrypt and decode the round's outputs on the client's behalf."""
        net = self.nets[req.net]
        r = req.client.round
        info = net.infos[r]
        res = np.zeros((info["n_groups"], self.L, self.n), dtype=np.uint64)
        sf.sf_decrypt(self.ctx, self.sks[req.key], req.d_out, info["n_groups"], res, self.stream)
        vals = nw.decode_outputs(net, r, res)
        if not np.all(np.abs(vals) < self.activation_bound):
            raise RuntimeError(f"request {req.rid} ({req.net}, key {req.key}) round {r}: decoded |value| "
                               f"{np.abs(vals).max():.3g} is not a plausible activation; engine call held "
                               f"{self.last_call}")
        req.client.absorb(r, vals, req.sigma_out)
        # the simulated client never loses a download here: nothing is kept to resend
        req.session.complete(r, None)
        req.down_bytes += protocol.round_bytes(info, self.L, self.n, net.gammas[r])[1]
        req.rounds_run += 1
        req.d_in = req.d_out = req.d_pow = None

    def evaluate(self, batch: list):
        """One engine call over the pending rounds of `batch`."""
        layers, rks, d_ins, d_pows, k_ins, sps, sos, d_outs, caps = [], [], [], [], [], [], [], [], []
        for req in batch:
            net = self.nets[req.net]
            r = req.client.round
            info = net.infos[r]
            layers.append(net.layers[r])
            rks.append(self.rks[req.key])
            d_ins.append(req.d_in)
            d_pows.append(req.d_pow)
            k_ins.append(info["k_in"])
            sps.append(req.sigma_prev)
            sos.append(req.sigma_out)
            d_outs.append(req.d_out)
            caps.append(info["n_groups"])
        self.last_call = [(req.rid, req.net, req.key, req.client.round) for req in batch]
        if any(d is not None for d in d_pows):
            sf.sf_eval_layers_gamma(self.ctx, layers, rks, d_ins, d_pows, k_ins, sps, sos, d_outs, caps, self.stream)
        else:
            sf.sf_eval_layers(self.ctx, layers, rks, d_ins, k_ins, sps, sos, d_outs, caps, self.stream)
        self.stream.synchronize()

    def destroy(self):
        for net in self.nets.values():
            net.destroy()
        for rk in self.rks:
            sf.sf_rotkeys_destroy(rk)
        for sk in self.sks:
            sf.sf_secret_key_destroy(sk)
        sf.sf_ctx_destroy(self.ctx)
        sf.sf_params_destroy(self.params)


class Server:
    """Admission queue + one continuous-batching worker per pool."""

    def __init__(self, pools: dict, route: dict, mem_budget: int, max_queue: int = 64, max_active=16,
                 max_batch: int = 32):
        self.pools = pools                 # pool name -> Pool
        self.route = route                 # network name -> pool name
        self.mem_budget = mem_budget
        self.max_queue, self.max_batch = max_queue, max_batch
        # requests a worker may hold: one number for every pool, or per pool
        self.max_active = max_active if isinstance(max_active, dict) else {p: max_active for p in pools}
        self.lock = threading.Condition()
        self.queue = collections.deque()
        self.inbox = {p: [] for p in pools}
        self.active = {p: [] for p in pools}
        self.held = {p: 0 for p in pools}     # admitted and not finished, per pool
        self.used = 0
        self.stop = False
        self.rejected, self.completed, self.admitted = [], [], []
        self.batches = []                  # (pool, rounds in the call, ms)
        self.errors = []
        self.threads = [threading.Thread(target=self._worker, args=(p,), daemon=True) for p in pools]

    def start(self):
        for t in self.threads:
            t.start()

    def submit(self, req: Request) -> bool:
        pool = self.pools[self.route[req.net]]
        req.arrival = time.perf_counter()
        req.reserve = pool.reserve_of(req.net)
        with self.lock:
            if len(self.queue) >= self.max_queue or req.reserve > self.mem_budget:
                self.rejected.append(req)
                return False
            self.queue.append(req)
            self._admit()
            self.lock.notify_all()
        return True

    def _admit(self):
        while self.queue:
            req = self.queue[0]
            p = self.route[req.net]
            if self.used + req.reserve > self.mem_budget or self.held[p] >= self.max_active[p]:
                break
            self.queue.popleft()
            self.used += req.reserve
            self.held[p] += 1
            req.admitted = time.perf_counter()
            req.client = self.pools[p].new_client(req)
            self.inbox[p].append(req)
            self.admitted.append(req)

    def _finish(self, p: str, req: Request):
        req.finished = time.perf_counter()
        req.logits = req.client.logits()
        with self.lock:
            self.used -= req.reserve
            self.held[p] -= 1
            self.completed.append(req)
            self._admit()
            self.lock.notify_all()

    def _worker(self, p: str):
        pool = self.pools[p]
        try:
            pool.bind_thread()
            while True:
                with self.lock:
                    while not self.stop and not self.inbox[p] and not self.active[p]:
                        self.lock.wait(timeout=0.05)
                    if self.stop:
                        return
                    new, self.inbox[p] = self.inbox[p], []
                for req in new:
                    pool.prepare(req)
                    self.active[p].append(req)
                batch = self.active[p][:self.max_batch]
                t0 = time.perf_counter()
                pool.evaluate(batch)
                self.batches.append((p, len(batch), (time.perf_counter() - t0) * 1e3))
                done = []
                for req in batch:
                    pool.absorb(req)
                    if req.client.done:
                        done.append(req)
                    else:
                        pool.prepare(req)
                for req in done:
                    self.active[p].remove(req)
                    self._finish(p, req)
                # rotate so that requests beyond max_batch get their turn
                if len(self.active[p]) > self.max_batch:
                    k = len(batch) - len(done)
                    self.active[p] = self.active[p][k:] + self.active[p][:k]
        except Exception as e:     # surfaced by shutdown()
            self.errors.append(repr(e))
            with self.lock:
                self.stop = True
                self.lock.notify_all()

    def idle(self) -> bool:
        with self.lock:
            return not self.queue and all(v == 0 for v in self.held.values())

    def shutdown(self):
        with self.lock:
            self.stop = True
            self.lock.notify_all()
        for t in self.threads:
            t.join()
        if self.errors:
            raise RuntimeError("server worker failed: " + "; ".join(self.errors))


def make_request(rid: int, net: str, key: int, seed: int) -> Request:
    return Request(rid, net, key, wl.network_input(net, seed), session_seed=seed * 7 + 1, request_seed=seed)


def poisson_arrivals(rate: float, duration: float, mix: dict, n_clients: int, seed: int) -> list:
    """(time offset, network, client key, request seed) for Poisson(rate)
    arrivals over `duration` seconds; networks drawn by the `mix` weights."""
    rng = np.random.default_rng(seed)
    names = list(mix)
    w = np.array([mix[k] for k in names], dtype=np.float64)
    w /= w.sum()
    t, out, i = 0.0, [], 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            return out
        out.append((t, names[int(rng.choice(len(names), p=w))], int(rng.integers(n_clients)), seed * 100000 + i))
        i += 1


def run_arrivals(server: Server, arrivals: list, drain: float, verify: bool = False) -> dict:
    """Replays the arrivals in real time, then waits up to `drain` seconds for
    admitted requests to finish.  Returns the run's statistics."""
    server.start()
    t0 = time.perf_counter()
    for i, (dt, net, key, seed) in enumerate(arrivals):
        now = time.perf_counter() - t0
        if dt > now:
            time.sleep(dt - now)
        server.submit(make_request(i, net, key, seed))
    window = time.perf_counter() - t0
    t_end = time.perf_counter() + drain
    while time.perf_counter() < t_end and not server.idle() and not server.errors:
        time.sleep(0.02)
    elapsed = time.perf_counter() - t0
    unfinished = len(server.admitted) - len(server.completed)
    server.shutdown()
    lat = np.array([r.finished - r.arrival for r in server.completed]) if server.completed else np.array([])
    rounds = sum(r.rounds_run for r in server.admitted)
    per_net = {}
    for net in sorted({r.net for r in server.admitted}):
        ln = np.array([r.finished - r.arrival for r in server.completed if r.net == net])
        per_net[net] = {"completed": int(ln.size),
                        "admitted": sum(1 for r in server.admitted if r.net == net),
                        "p50_latency_s": float(np.percentile(ln, 50)) if ln.size else None,
                        "p99_latency_s": float(np.percentile(ln, 99)) if ln.size else None}
    errs = {}
    if verify:
        # every completed request against the plaintext network in float64
        for req in server.completed:
            net = server.pools[server.route[req.net]].nets[req.net]
            e = float(np.abs(req.logits - nw.float_forward(net, req.x)).max())
            errs[req.net] = max(errs.get(req.net, 0.0), e)
    return {"arrivals": len(arrivals), "admitted": len(server.admitted), "rejected": len(server.rejected),
            "max_abs_err_vs_float64": errs if verify else None,
            "completed": len(server.completed), "unfinished_at_end": unfinished,
            "rejection_rate": len(server.rejected) / max(1, len(arrivals)),
            "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
            "layers_per_s": rounds / elapsed, "rounds_run": rounds, "window_s": window, "elapsed_s": elapsed,
            "engine_calls": len(server.batches),
            "bytes_up": sum(r.up_bytes for r in server.admitted),
            "bytes_down": sum(r.down_bytes for r in server.admitted),
            "mean_rounds_per_call": float(np.mean([b[1] for b in server.batches])) if server.batches else None,
            "per_network": per_net}


SERVE_MIX = {"resnet20": 0.7, "resnet18": 0.3}


def bench(args, device: int) -> int:
    """Serving measurement: ResNet-20 requests at N = 2^14 (3 x 50-bit + 1)
    and ResNet-18 requests at N = 2^15 (4 x 50-bit + 2), 70/30, 4 client keys,
    Poisson arrivals at each rate of --rates for --duration seconds, then up to
    --drain seconds for admitted requests to finish.  Beside it, one ResNet-20
    request alone with one engine call per round (the plain form)."""
    import torch
    torch.cuda.set_device(device)
    gamma = getattr(args, "gamma", 0)
    pools = {"c2": Pool(wl.PARAMS["conv16"], ["resnet20"], 4, device, key_seed=7000, priority=-1, gamma=gamma),
             "c3": Pool(wl.PARAMS["r18"], ["resnet18"], 4, device, key_seed=8000, priority=0, gamma=gamma)}
    route = {"resnet20": "c2", "resnet18": "c3"}
    budget = 48 << 30
    max_active = {"c2": 16, "c3": 2}
    out = {"metric": "served encrypted layers/s; p50/p99 latency", "unit": "layers/s", "workload": "serve",
           "gamma": gamma,
           "mix": SERVE_MIX, "client_keys": 4, "mem_budget_bytes": budget, "max_active": max_active,
           "stream_priority": {"c2": -1, "c3": 0},
           "duration_s": args.duration, "drain_s": args.drain, "rates": {}}
    srv = Server({"c2": pools["c2"]}, {"resnet20": "c2"}, budget, max_active=1, max_batch=1)
    stats = run_arrivals(srv, [(0.0, "resnet20", 0, 99)], drain=600.0)
    out["alone"] = {"resnet20": {"latency_s": stats["p50_latency_s"], "layers_per_s": stats["layers_per_s"]}}
    for rate in [float(r) for r in args.rates.split(",")]:
        arr = poisson_arrivals(rate, args.duration, SERVE_MIX, 4, seed=int(rate * 1000) + 17)
        srv = Server(pools, route, budget, max_active=max_active)
        out["rates"][str(rate)] = run_arrivals(srv, arr, args.drain, verify=True)
    # below capacity: ResNet-20 requests alone at a low rate
    if args.low_rate > 0:
        arr = poisson_arrivals(args.low_rate, args.low_duration, {"resnet20": 1.0}, 4, seed=31)
        srv = Server({"c2": pools["c2"]}, {"resnet20": "c2"}, budget, max_active=16)
        out["resnet20_only"] = dict(rate=args.low_rate, duration_s=args.low_duration,
                                    **run_arrivals(srv, arr, args.drain, verify=True))
    for p in pools.values():
        p.destroy()
    print(json.dumps(out), flush=True)
    return 0
