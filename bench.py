"""Benchmark: encrypted linear layers per second on one GB300 (or N replicas).

One step = one full server round of the benchmark layer through the C ABI
(sf_eval_linear_layer).  The default layer (``--workload r34``) is a round of
the ResNet-34-shaped network at the largest parameter set: the first conv of
its last stage, 3x3 stride 2, 256 -> 512 channels on a 14x14x256 input, ring
N = 2^16 with 5 x 50-bit data primes and 2 special primes, fixed-point scale
2^40, with the input unshuffle and the output shuffle: 25088 leaf products
over 2304 taps each, 32767 pack-tree merges and 1 trace step (32768
automorphism + hybrid key switches), 1 packed output ciphertext.
``--workload conv16`` is the ResNet-20 stage-1 conv (3x3, 16 -> 16 on
16x32x32) at N = 2^14 with 3 x 50-bit + 1 special prime.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload r34|conv16|resnet18|resnet34|serve] [--no-extras]

The one-layer workloads print the one-line benchmark record.  Unless
--no-extras is given, the r34 line also carries, measured after its timed
region: the conv16 round (``conv16``), a bounded serving run of ResNet-20
requests below capacity with p50/p99 latency (``serving``), and the last five
rounds of the ResNet-18 network at N = 2^15 as one batched call against one
call per round (``batched_vs_per_layer``).  The other workloads are the
network-scale measurements, each one JSON line: resnet18 (all 18 layer rounds
of a ResNet-18 on 3x64x64 at N = 2^15, each with its own synthetic input: one
sf_eval_layers batch vs one call per layer), resnet34 (every round of a
ResNet-34 on 3x224x224 at N = 2^16, per layer and end to end) and serve
(Poisson arrivals of encrypted ResNet-20 / ResNet-18 requests through the
continuous-batching server).

--impl reference times the CPU oracle (the plain schoolbook implementation
under oracle/) on the host cores, on a bounded sample of the same layer
extrapolated to whole layers.  Under torchrun each rank runs an independent
replica (the round has no cross-GPU exchange); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted linear layers/s"
UNIT = "layers/s"
LAYERS = {
    # name: (parameter set, case factory name, keygen / encrypt / rotation-key seeds, description)
    "r34": ("r34", ("resnet34", "s3b0c1", 401), (403, 404, 405),
            "r34.s3b0c1: ResNet-34 conv 3x3 stride 2, 256 -> 512 channels on 14x14x256 (E = 50176, "
            "E' = 25088, 2304 taps per output), N = 2^16, 5 x 50-bit + 2 special primes, scale 2^40, input "
            "unshuffle + output shuffle, 1 packed output of 32768 slots, 32768 key switches per layer"),
    "conv16": ("conv16", None, (203, 204, 205),
               "conv16: ResNet-20 conv 3x3 16->16 on 16x32x32 (E = E' = 16384), N = 2^14, 3 x 50-bit + 1 "
               "special prime, scale 2^40, input unshuffle + output shuffle, 2 packed outputs of 8192, "
               "16384 key switches per layer"),
}
WORKLOAD = LAYERS["r34"][3]
NTT_POLYS = 512        # forward-NTT record: 512 x L limbs of the benchmark ring
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch batch")
    ap.add_argument("--reference-sample-s", type=float, default=8.0,
                    help="--impl reference: CPU seconds bound of each step's oracle sample")
    ap.add_argument("--workload", default="r34", choices=["r34", "conv16", "resnet18", "resnet34", "serve"])
    ap.add_argument("--gamma", type=int, default=0, choices=[0, 2],
                    help="resnet34 / serve: partial trace extraction level of every round (Sec. 4.3, 4.4)")
    ap.add_argument("--gamma-plan", action="store_true",
                    help="resnet34: a gamma = 0 calibration request with the kernel split, then the "
                         "timed request with the per-round levels the planner picks")
    ap.add_argument("--no-extras", action="store_true",
                    help="r34: skip the conv16, serving and batched-vs-per-layer sub-records")
    ap.add_argument("--rates", default="5,20,200", help="serve: arrival rates (requests/s)")
    ap.add_argument("--duration", type=float, default=20.0, help="serve: arrival window per rate (s)")
    ap.add_argument("--drain", type=float, default=60.0, help="serve: time allowed after the window (s)")
    ap.add_argument("--low-rate", type=float, default=0.3, help="serve: ResNet-20-only rate below capacity (0 = skip)")
    ap.add_argument("--low-duration", type=float, default=30.0, help="serve: window of the low-rate run (s)")
    ap.add_argument("--ctx-opt", action="append", default=[],
                    help="context option NAME=VALUE for the measured context (sf_ctx_set_option)")
    ap.add_argument("--layer-stats", default="",
                    help="resnet18/resnet34: only a per-kernel breakdown of these rounds (comma-separated names)")
    ap.add_argument("--small", action="store_true",
                    help="profiling case: the same kernel shapes on a smaller layer (conv16: 8x16x16, 2048 "
                         "outputs; r34: 64x7x7 -> 256 channels, 12544 outputs; a few GB on the device)")
    return ap.parse_args()


# --------------------------------------------------------------- clocks ----

class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ workload ----

class Workload:
    """Keys, weights and the encrypted input of a benchmark layer, resident on the device."""

    def __init__(self, device: int, kind: str = "r34", small: bool = False):
        import torch
        import paper_2509_01253_gb300 as sf
        from paper_2509_01253_gb300 import workloads as wl
        self.sf, self.torch = sf, torch
        pset, case_of, (s_key, s_enc, s_rot), desc = LAYERS[kind]
        self.kind, self.desc = kind, desc
        self.ps = ps = wl.PARAMS[pset]
        if kind == "conv16":
            self.case = case = wl.small_conv_case(201, 8, 16, 16, 16) if small else wl.conv16_case()
        elif small:
            self.case = case = wl.small_conv_case(401, 7, 7, 64, 256, x_range=(0.0, 1.0))
        else:
            self.case = case = wl.round_case(*case_of)
        if small:
            self.desc = f"{kind}-small (profiling case, same ring and kernels): {case.name}, E' = {case.E_out}"
        self.params = sf.sf_params_create(ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits, ps.sigma)
        self.ctx = sf.sf_ctx_create(self.params, device)
        self.sk = sf.sf_keygen(self.ctx, s_key)
        self.rk = sf.sf_gen_rotation_keys(self.ctx, self.sk, None, s_rot)
        W = np.concatenate([w.ravel() for w in case.weights])
        self.layer = sf.sf_encode_weights(self.ctx, case.terms, W, None, ps.delta, ps.delta ** 2)
        self.info = sf.sf_layer_get_info(self.ctx, self.layer)
        self.n, self.L = 1 << ps.log_n, ps.n_data
        xs = case.x if case.sigma_prev is None else case.x[case.sigma_prev.astype(np.int64)]
        self.msg = sf.sf_encode_input(xs, ps.delta)
        self.k_in, self.G = self.info["k_in"], self.info["n_groups"]
        dev = f"cuda:{device}"
        self.d_in = torch.zeros((self.k_in, 2, self.L, self.n), dtype=torch.int64, device=dev)
        sf.sf_encrypt(self.ctx, self.sk, self.msg, s_enc, self.d_in, self.k_in)
        self.d_out = torch.zeros((self.G, 2, self.L, self.n), dtype=torch.int64, device=dev)
        self.stream = torch.cuda.current_stream(device)
        self.ct_bytes = 2 * self.L * self.n * 8

    def destroy(self):
        sf = self.sf
        sf.sf_layer_destroy(self.layer)
        sf.sf_rotkeys_destroy(self.rk)
        sf.sf_secret_key_destroy(self.sk)
        sf.sf_ctx_destroy(self.ctx)
        sf.sf_params_destroy(self.params)
        self.d_in = self.d_out = None

    def step(self):
        self.sf.sf_eval_linear_layer(self.ctx, self.layer, self.rk, self.d_in, self.k_in, self.case.sigma_prev,
                                     self.case.sigma_out, self.d_out, self.G, self.stream)

    def autotune(self):
        """The library's autotuner on this layer: keeps the fastest key-switch
        launch batch and leaf column pass in the context."""
        best, ms = self.sf.sf_autotune_layers(self.ctx, [self.layer], [self.rk], [self.d_in], [self.k_in],
                                              [self.case.sigma_prev], [self.case.sigma_out], [self.d_out], [self.G],
                                              2, self.stream)
        return {"ks_batch": best, "ms": ms,
                "ks3_threads": self.sf.sf_ctx_get_option(self.ctx, "ks3_threads"),
                "leaf_sparse": self.sf.sf_ctx_get_option(self.ctx, "leaf_sparse"),
                "row_radix": self.sf.sf_ctx_get_option(self.ctx, "row_radix")}

    def check(self) -> float:
        """Max |decoded - float64| over all outputs (not timed)."""
        from paper_2509_01253_gb300 import workloads as wl
        sf = self.sf
        sf.sf_sync(self.ctx, self.stream)
        res = np.zeros((self.G, self.L, self.n), dtype=np.uint64)
        sf.sf_decrypt(self.ctx, self.sk, self.d_out, self.G, res, self.stream)
        vals = sf.sf_decode(self.params, res, self.G, self.n // self.info["group_size"], self.info["E_out"],
                            self.ps.delta ** 2)
        ref = wl.float_reference(self.case)
        if self.case.sigma_out is not None:
            ref = ref[self.case.sigma_out.astype(np.int64)]
        return float(np.abs(vals - ref).max())


def flush_l2(buf):
    buf.add_(1)


def launches(sf, ctx) -> dict:
    return {name: (cnt, ms) for name, cnt, ms in sf.sf_kernel_stats(ctx)}


# ------------------------------------------------------------ roofline ----

class RingShape:
    """Sizes the work model needs: N = R x C split, moduli counts, digits."""

    def __init__(self, p_info: dict):
        self.n = p_info["n"]
        self.L, self.K, self.dnum = p_info["n_data"], p_info["n_special"], p_info["dnum"]
        self.nm = self.L + self.K
        log_n = self.n.bit_length() - 1
        # the library's split N = R x C (2^16 = 128 x 512)
        self.lc = 9 if log_n == 16 else (log_n + 1) // 2
        self.lr = log_n - self.lc
        self.digits = [min(self.K, self.L - j * self.K) for j in range(self.dnum)]


def kernel_ops(kernel: str, g: RingShape, k_in: int = 1):
    """Modular multiplications of one item of a kernel, split by kind:
    (forward butterflies, inverse butterflies, other products: monomial and
    key multiply-accumulates, base conversions, scalings).  Items are merges
    (key switches) for the ks* kernels, (output, input ciphertext) pairs for
    leaf_col and outputs for leaf_row.  A one-limb ModUp digit converts with
    no product (its residue is the value), and the ModDown factor P^-1 rides
    on the key and the conversion constants, so the finish has no product."""
    N, L, K, nm, dnum, lr, lc = g.n, g.L, g.K, g.nm, g.dnum, g.lr, g.lc
    half = N // 2
    fbc_up = sum(d * (nm - d) for d in g.digits if d > 1) * N
    ext = dnum * nm - L   # digit extensions: every modulus outside the digit
    table = {
        "ks_gather": (0, 0, 4 * L * N),
        "ks1_inv_row": (0, L * half * lc, 0),
        "ks2_modup_col": (ext * half * lr, L * half * lr, L * N + fbc_up),
        "ks3_inner_row": (ext * half * lc, 0, 2 * dnum * nm * N),
        "ks3_inv_row_p": (0, 2 * K * half * lc, 0),
        "ks4_moddown_col": (2 * L * half * lr, 2 * K * half * lr, 2 * K * N + 2 * K * L * N),
        "ks5_finish_row": (2 * L * half * lc, 0, 0),
        "leaf_col": (L * half * lr, 0, 0),
        "leaf_row": (k_in * L * half * lc, 0, 2 * k_in * L * N),
    }
    return table.get(kernel)


def kernel_work(kernel: str, g: RingShape, k_in: int = 1):
    """Algorithmic work of one item of a kernel: (HBM bytes, modular
    multiplications), items as in kernel_ops.  Bytes are the operands that
    must cross HBM in the kernel's stage of the pipeline (one read of each
    input limb, one write of each output limb, 8-byte words; the rotation key
    is read once per launch and not counted per item); a modular
    multiplication is one butterfly, one multiply-accumulate or one
    base-conversion product."""
    N, L, K, nm, dnum, w = g.n, g.L, g.K, g.nm, g.dnum, 8
    nbytes = {
        # read E and O (both parts), write TA and the merge's v + tau(u.b)
        "ks_gather": 7 * L * N * w,
        "ks1_inv_row": 2 * L * N * w,
        "ks2_modup_col": dnum * nm * N * w,
        "ks3_inner_row": (dnum * nm + 2 * nm) * N * w,
        "ks3_inv_row_p": 4 * K * N * w,
        "ks4_moddown_col": (2 * K + 2 * L) * N * w,
        # read conv, acc and out (2L limbs each), write out
        "ks5_finish_row": 8 * L * N * w,
        "leaf_col": L * N * w,
        "leaf_row": (k_in * L + 2 * L) * N * w,
    }.get(kernel)
    ops = kernel_ops(kernel, g, k_in)
    if nbytes is None or ops is None:
        return None
    return nbytes, sum(ops)


def probe_ceiling(ops, probe):
    """Arithmetic ceiling of a kernel's mix of operations from the measured
    per-kind rates (Gmodmul/s): total / sum(count_k / rate_k)."""
    if not probe or not ops or sum(ops) == 0:
        return None
    t = ops[0] / probe["fwd_bfly"] + ops[1] / probe["inv_bfly"] + ops[2] / probe["mac"]
    return sum(ops) / t


def alu_peak(sm_count: int, sm_mhz: float):
    """Modular-multiplication peak from unit counts and clock: 64 32-bit
    integer multiply-adds per clock per SM, and 10 of them per 64-bit Shoup
    product (3 for each of the two low 64-bit products, 4 for the high one)."""
    return sm_count * 64 * sm_mhz * 1e6 / 10.0


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    except (OSError, ValueError):
        return 6800.0, "fallback"


# per-item DRAM bytes (read + write) of a kernel at a ring size (log2 N), from
# an ncu capture of a small case of the same kernel and ring
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch divided by its
# items), kept only while the kernel's code is unchanged since the capture;
# scaled to a full launch by its items
TRAFFIC_PER_ITEM = {
    # k_ks3 at N = 2^16 (5 + 2 primes), 128 x 512 split: one launch of 128
    # merges of the small r34 case (--small, ks_batch=128), 1.636432 GB read +
    # 0.849524 GB written
    ("ks3_inner_row", 16): (1.636432e9 + 0.849524e9) / 128,
}


def items_per_layer(kernel: str, info: dict, merges: int) -> int:
    if kernel.startswith("ks"):
        return merges
    if kernel == "leaf_col":
        return info["E_out"] * info["k_in"]
    if kernel == "leaf_row":
        return info["E_out"]
    return 0


def roofline_of(kstats: dict, k_steps: int, g: RingShape, info: dict, total_kernel_ms: float, clk: dict,
                merges: int = None, probe: dict = None, sm_count: int = 152):
    """Roofline record of the kernel with the largest device-time share:
    algorithmic work per layer / its measured time per layer, against the
    measured HBM copy bandwidth and the derived modular-multiplication peak;
    `bound` is the one whose time at peak is larger."""
    merges = info["ks_count"] if merges is None else merges
    top = max((k for k in kstats if kernel_work(k, g, info["k_in"])), key=lambda k: kstats[k][1])
    cnt, ms = kstats[top]
    per_layer_s = ms / k_steps / 1e3
    items = items_per_layer(top, info, merges)
    b_item, m_item = kernel_work(top, g, info["k_in"])
    hbm_peak, peak_kind = load_peaks()
    alu_pk = alu_peak(sm_count, 2070.0)
    hbm_ach = b_item * items / per_layer_s / 1e9
    alu_ach = m_item * items / per_layer_s / 1e9
    t_hbm = b_item / (hbm_peak * 1e9)
    t_alu = m_item / alu_pk
    bound = "alu" if t_alu >= t_hbm else "hbm"
    ceil = probe_ceiling(kernel_ops(top, g, info["k_in"]), probe)
    launches = cnt // k_steps
    traffic = TRAFFIC_PER_ITEM.get((top, g.n.bit_length() - 1))
    rec = {"bound": bound, "kernel": top,
           "achieved": alu_ach if bound == "alu" else hbm_ach,
           "peak": alu_pk / 1e9 if bound == "alu" else hbm_peak,
           "unit": "Gmodmul/s" if bound == "alu" else "GB/s"}
    rec["frac"] = rec["achieved"] / rec["peak"]
    rec["traffic"] = traffic * items / launches if traffic else None
    rec.update({
        "peak_source": (f"derived: {sm_count} SMs x 64 int32 multiply-adds/clk x 2070 MHz / 10 per 64-bit modmul"
                        if bound == "alu" else f"{peak_kind} hbm_gbs"),
        "hbm_view": {"achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_ach / hbm_peak,
                     "peak_source": peak_kind},
        "alu_view": {"achieved": alu_ach, "peak": alu_pk / 1e9, "unit": "Gmodmul/s", "frac": alu_ach * 1e9 / alu_pk,
                     "at_median_clock": (alu_ach * 1e9 / alu_peak(sm_count, clk["sm_mhz"])) if clk.get("sm_mhz") else None,
                     "probe_peak": ceil, "frac_of_probe": (alu_ach / ceil) if ceil else None,
                     "probe_source": "sf_modmul_probe: register-resident butterflies and multiply-accumulates "
                                     "measured on this GPU, weighted by this kernel's mix of operations"},
        "algorithmic_bytes_per_launch": b_item * items / launches,
        "algorithmic_modmul_per_launch": m_item * items / launches,
        "avg_launch_us": per_layer_s / launches * 1e6, "launches_per_layer": launches,
        "share_of_device_time": ms / total_kernel_ms if total_kernel_ms else None})
    return rec


def measure_probe(sf, ctx) -> dict:
    """Measured arithmetic ceilings (Gmodmul/s) of the library's forward and
    inverse butterflies and key multiply-accumulates on this GPU."""
    return {"fwd_bfly": sf.sf_modmul_probe(ctx, 0), "inv_bfly": sf.sf_modmul_probe(ctx, 1),
            "mac": sf.sf_modmul_probe(ctx, 2), "unit": "Gmodmul/s"}


def ntt_record(sf, torch, wl_, p_info: dict, probe: dict, flush) -> dict:
    """Batched forward NTT of every limb of NTT_POLYS polynomials of the
    benchmark ring (sf_ntt_batch, inputs and outputs larger than L2):
    algorithmic GB/s (each limb read once and written once) against the
    measured HBM bandwidth, and butterflies/s against the measured forward
    butterfly ceiling."""
    L, n = wl_.L, wl_.n
    count = NTT_POLYS
    qmin = min(p_info["moduli"][:L])
    dev = wl_.d_in.device
    x = torch.randint(0, qmin, (count, L, n), dtype=torch.int64, device=dev)
    y = torch.empty_like(x)
    stream = wl_.stream
    for _ in range(3):
        sf.sf_ntt_batch(wl_.ctx, x, y, count, False, stream)
    reps = 5
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for i in range(reps):
        flush_l2(flush)
        ev[i][0].record(stream)
        sf.sf_ntt_batch(wl_.ctx, x, y, count, False, stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / reps
    limbs = count * L
    nbytes = 2 * limbs * n * 8
    bfly = limbs * (n // 2) * (n.bit_length() - 1)
    hbm_peak, kind = load_peaks()
    gbs = nbytes / (ms * 1e-3) / 1e9
    gmm = bfly / (ms * 1e-3) / 1e9
    return {"what": f"forward NTT of {count} x {L} limbs of N = {n} (sf_ntt_batch, two persistent passes)",
            "ms_per_call": ms, "algorithmic_bytes": nbytes, "gbs": gbs, "hbm_peak": hbm_peak, "peak_source": kind,
            "frac_hbm": gbs / hbm_peak, "gmodmul_s": gmm, "frac_of_probe": gmm / probe["fwd_bfly"]}


def pp_ntt_record(local: int, flush, t: int = 3, alpha: int = 7, L: int = 5, count: int = 4096) -> dict:
    """Batched length-M transform of the paper's prime-power ring M = 3^7
    (Table 2; sf_pp_ntt, one block per limb, radix-3 stages in shared memory)
    over count x L limbs: algorithmic GB/s (each limb read and written once)
    and modular products/s: M/t butterflies per stage, alpha stages, each
    with its t - 1 twiddle products and the t-point DFT's products (2 for
    t = 3, (t - 1)^2 / 2 by conjugate pairs otherwise)."""
    import torch
    import paper_2509_01253_gb300 as sf
    r = sf.sf_pp_ring_create(t, alpha, L, 50, local)
    try:
        info = sf.sf_pp_ring_info(r, L)
        M = info["M"]
        x = torch.randint(0, min(info["moduli"]), (count, L, M), dtype=torch.int64, device=f"cuda:{local}")
        y = torch.empty_like(x)
        stream = torch.cuda.current_stream()
        for _ in range(3):
            sf.sf_pp_ntt(r, x, y, count, False, stream)
        reps = 5
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for i in range(reps):
            flush_l2(flush)
            ev[i][0].record(stream)
            sf.sf_pp_ntt(r, x, y, count, False, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / reps
        nbytes = 2 * count * L * M * 8
        mods = count * L * (M // t) * alpha * ((2 if t == 3 else (t - 1) ** 2 // 2) + t - 1)
        hbm_peak, kind = load_peaks()
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"what": f"forward length-{M} transform (M = {t}^{alpha}, N = {info['N']}) of {count} x {L} limbs "
                        f"(sf_pp_ntt)", "ms_per_call": ms, "algorithmic_bytes": nbytes, "gbs": gbs,
                "frac_hbm": gbs / hbm_peak, "peak_source": kind, "gmodmul_s": mods / (ms * 1e-3) / 1e9}
    finally:
        sf.sf_pp_ring_destroy(r)


def tq_record(local: int, flush, count: int = 4096) -> dict:
    """The paper's torus scheme (q = 2^53) with Table 2's rings and gadgets:
    one sf_tq_keyswitch launch over `count` ciphertexts per gadget (one fused
    kernel: tau_h, gadget digits, 2 (l + 2) length-M transforms over two CRT
    primes, the key products and the CRT), and the full homomorphic trace of
    `count` ciphertexts at M = 5^5, (310, 5).  Modular products per key switch,
    counted nominally: per transform alpha stages of M / t butterflies with the
    DFT's products (2 at t = 3, (t - 1)^2 / 2 otherwise) and t - 1 twiddles;
    per prime 2 l M key products and 2 M inverse scalings; 2 N CRT steps of two
    products each.  Inputs are larger than L2 (4096 x 2 x N words) and L2 is
    flushed before every timed call."""
    import torch
    import paper_2509_01253_gb300 as sf
    dev = f"cuda:{local}"
    stream = torch.cuda.current_stream()
    alu_pk = alu_peak(torch.cuda.get_device_properties(local).multi_processor_count, 2070.0) / 1e9
    rows = []

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for i in range(reps):
            flush_l2(flush)
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / reps

    def setup(t, alpha, D, l, h_of=None):
        r = sf.sf_tq_ring_create(t, alpha, D, l, local)
        info = sf.sf_tq_ring_info(r)
        N = info["N"]
        g = torch.Generator(device=dev).manual_seed(11)
        s = torch.randint(-1, 2, (N,), dtype=torch.int64, device=dev, generator=g)
        a = torch.randint(0, 2 ** 53, (count, N), dtype=torch.int64, device=dev, generator=g)
        m = torch.randint(0, 2 ** 53, (count, N), dtype=torch.int64, device=dev, generator=g)
        e = torch.randint(-2 ** 17, 2 ** 17, (count, N), dtype=torch.int64, device=dev, generator=g)
        ct = torch.empty((count, 2, N), dtype=torch.int64, device=dev)
        sf.sf_tq_encrypt(r, s, a, m, e, ct, count, stream)
        return r, info, s, ct, g

    def key(r, info, s, h, l, g):
        N = info["N"]
        ka = torch.randint(0, 2 ** 53, (l, N), dtype=torch.int64, device=dev, generator=g)
        ek = torch.randint(-2 ** 17, 2 ** 17, (l, N), dtype=torch.int64, device=dev, generator=g)
        kb = torch.empty_like(ka)
        sf.sf_tq_ksk(r, s, h, ka, ek, kb, stream)
        k = torch.empty(info["key_words"], dtype=torch.int64, device=dev)
        sf.sf_tq_key_prepare(r, ka, kb, k, stream)
        return k

    def products(t, alpha, M, N, l):
        per_tr = alpha * (M // t) * ((2 if t == 3 else (t - 1) ** 2 // 2) + t - 1)
        return 2 * (l + 2) * per_tr + 2 * (2 * l * M + 2 * M) + 2 * 2 * N

    for t, alpha, D, l in ((3, 7, 512, 3), (7, 4, 2 ** 12, 3), (7, 4, 2 ** 16, 2), (5, 5, 310, 5), (5, 5, 310, 4)):
        r, info, s, ct, g = setup(t, alpha, D, l)
        try:
            M, N = info["M"], info["N"]
            h = 1 + t ** (alpha - 1)
            k = key(r, info, s, h, l, g)
            out = torch.empty_like(ct)
            ms = timed(lambda: sf.sf_tq_keyswitch(r, ct, out, count, h, k, stream))
            prods = products(t, alpha, M, N, l) * count
            gm = prods / (ms * 1e-3) / 1e9
            rows.append({"M": f"{t}^{alpha}", "N": N, "D": D, "l": l, "ciphertexts": count, "ms_per_call": ms,
                         "us_per_keyswitch": ms * 1e3 / count, "keyswitches_per_s": count / (ms * 1e-3),
                         "gmodmul_s": gm, "frac_alu_peak": gm / alu_pk,
                         "hbm_bytes": 2 * count * 2 * N * 8,
                         "gbs": 2 * count * 2 * N * 8 / (ms * 1e-3) / 1e9})
        finally:
            sf.sf_tq_ring_destroy(r)
        torch.cuda.empty_cache()
    # Tr_(K / K_1) at M = 5^5 with Table 2's gamma >= 1 gadget (310, 4): the
    # tower steps tau_(1 + 5^i), i = 4 .. 1, four key switches each
    r, info, s, ct, g = setup(5, 5, 310, 4)
    try:
        keys = {1 + 5 ** i: key(r, info, s, 1 + 5 ** i, 4, g) for i in range(1, 5)}
        out = torch.empty_like(ct)
        n_ks = sf.sf_tq_hom_trace(r, ct, out, count, 1, keys, stream)
        ms = timed(lambda: sf.sf_tq_hom_trace(r, ct, out, count, 1, keys, stream), reps=3)
        trace = {"what": f"Tr_(K/K_1) (gamma = 1) of {count} ciphertexts, M = 5^5, (D, l) = (310, 4)",
                 "keyswitches_per_ciphertext": n_ks, "ms_per_call": ms, "us_per_ciphertext": ms * 1e3 / count}
    finally:
        sf.sf_tq_ring_destroy(r)
    return {"what": "torus RLWE (q = 2^53) gadget key switch, Table 2's rings and gadgets (sf_tq_keyswitch)",
            "alu_peak_gmodmul_s": alu_pk, "peak_source": "derived: SMs x 64 int32 multiply-adds/clk x 2070 MHz / 10",
            "rows": rows, "trace": trace}


# ------------------------------------------------------- CPU baseline ----

def host_cores() -> int:
    cores = os.cpu_count()
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        pass
    omp = os.environ.get("OMP_NUM_THREADS")
    if omp:
        cores = min(cores, int(omp))
    return cores


class OracleSample:
    """The oracle on a bounded sample of a benchmark layer, on the host cores.

    Set-up (outside any timing): parameters, secret key, the encrypted layer
    input and the quantised layer.  Each sample times (a) leaf outputs, one
    output's extraction + unshuffle + linear step over all its taps at full
    size (oracle.linear_output), and (b) one schoolbook negacyclic limb product
    at full size per host core, run concurrently (oracle.polymul; ctypes
    releases the interpreter lock).  A layer is then E' leaf outputs plus
    ks_count key switches of 2 * dnum * (L + K) limb products each (the
    oracle's inner product with the key, spread over the host cores); the
    key switch's base conversions, automorphism and the packing additions
    (O(N) work each) are not counted, so the estimate is a lower bound on the
    oracle's time per layer."""

    def __init__(self, kind: str = "r34"):
        import oracle as O
        from paper_2509_01253_gb300 import workloads as wl
        self.O = O
        pset, case_of, (s_key, s_enc, _), _ = LAYERS[kind]
        ps = wl.PARAMS[pset]
        self.case = case = wl.conv16_case() if kind == "conv16" else wl.round_case(*case_of)
        self.prm = prm = O.make_params(ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits)
        s_o = O.keygen(prm, s_key)
        xs = case.x if case.sigma_prev is None else case.x[case.sigma_prev.astype(np.int64)]
        self.k_in = -(-xs.size // prm.n)
        self.cts = O.encrypt(prm, s_o, O.quantize(xs, ps.delta), s_enc, self.k_in)
        terms = [O.ConvTerm(t.in_offset, t.H, t.W, t.C_in, t.C_out, t.kh, t.kw, t.stride, t.pad) for t in case.terms]
        self.lay = O.make_layer(terms, case.weights, None, ps.delta, ps.delta ** 2)
        self.e_out = self.lay.E_out
        self.ks = O.ks_count(prm, self.e_out)
        self.prods_per_ks = 2 * prm.dnum * (prm.L + prm.K)
        self.cores = host_cores()
        rng = np.random.default_rng(7)
        q0 = prm.q[0]
        self.pa = [rng.integers(0, q0, prm.n, dtype=np.uint64) for _ in range(self.cores)]
        self.pb = [rng.integers(0, q0, prm.n, dtype=np.uint64) for _ in range(self.cores)]
        self.name = kind

    def run(self, max_seconds: float = 8.0):
        """Returns (layers/s, description) of one bounded sample."""
        from concurrent.futures import ThreadPoolExecutor
        O, case = self.O, self.case
        t0 = time.perf_counter()
        n_leaf = 0
        while True:
            o = int(case.sigma_out[n_leaf % self.e_out]) if case.sigma_out is not None else n_leaf % self.e_out
            O.linear_output(self.prm, self.lay, self.cts, o, case.sigma_prev)
            n_leaf += 1
            if n_leaf >= 8 or time.perf_counter() - t0 > max_seconds / 3:
                break
        t_leaf = (time.perf_counter() - t0) / n_leaf
        q0 = self.prm.q[0]
        with ThreadPoolExecutor(self.cores) as ex:
            t0 = time.perf_counter()
            list(ex.map(lambda i: O.polymul(self.pa[i], self.pb[i], q0), range(self.cores)))
            t_batch = time.perf_counter() - t0
        t_ks = self.prods_per_ks / self.cores * t_batch
        t_layer = self.e_out * t_leaf + self.ks * t_ks
        desc = (f"{self.name} layer at full size: {n_leaf} leaf outputs ({t_leaf:.3f} s each, x{self.e_out}) and "
                f"{self.cores} concurrent limb products of N = {self.prm.n} ({t_batch:.2f} s), i.e. "
                f"{t_ks:.2f} s per key switch of {self.prods_per_ks} limb products on {self.cores} cores "
                f"(x{self.ks}); base conversions, automorphisms and packing additions not counted; "
                f"extrapolated to one layer")
        return 1.0 / t_layer, desc


def oracle_sample(kind: str = "r34", max_seconds: float = 20.0):
    """One bounded oracle sample of the benchmark layer: (layers/s, cores, description)."""
    smp = OracleSample(kind)
    v, desc = smp.run(max_seconds)
    return v, smp.cores, desc


# ----------------------------------------------------------------- main ----

def max_over_ranks(dist, x: float) -> float:
    """The slowest rank's time (replicas run independently; only timings meet)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def replicas_value(ws: int, steps: int, total_s: float) -> float:
    """Whole-job throughput: every rank ran `steps` layer rounds; the job took the slowest rank's time."""
    return ws * steps / total_s


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        return dist, ws, rank, local
    return None, 1, 0, 0


def run_reference(args, dist, ws, rank):
    if rank != 0:
        return 0
    kind = args.workload if args.workload in LAYERS else "r34"
    smp = OracleSample(kind)
    times = []
    desc = None
    for i in range(args.warmup + args.steps):
        v, desc = smp.run(max_seconds=args.reference_sample_s)
        if i >= args.warmup:
            times.append(1.0 / v)
    sec = sum(times) / len(times)
    value = 1.0 / sec
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "impl": "reference",
            "config": {"workload": LAYERS[kind][3], "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": smp.cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------- network workloads ----

NET_PARAMS = {"resnet18": "r18", "resnet34": "r34", "resnet20": "conv16"}


class NetworkWorkload:
    """Every round of a network, each with its own seeded synthetic input
    (U(0, 1), a post-ReLU activation), input and output permutations drawn
    from the session seed (none before the first and after the last round),
    encrypted and resident on the device."""

    def __init__(self, kind: str, device: int, seed: int, names=None):
        import torch
        import paper_2509_01253_gb300 as sf
        from paper_2509_01253_gb300 import network as nw
        from paper_2509_01253_gb300 import workloads as wl
        self.sf, self.torch = sf, torch
        self.kind = kind
        self.ps = ps = wl.PARAMS[NET_PARAMS[kind]]
        self.params = sf.sf_params_create(ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits, ps.sigma)
        self.ctx = sf.sf_ctx_create(self.params, device)
        self.sk = sf.sf_keygen(self.ctx, seed + 3)
        self.rk = sf.sf_gen_rotation_keys(self.ctx, self.sk, None, seed + 5)
        rounds = wl.resnet_rounds(kind)
        if names is not None:
            rounds = [r for r in rounds if r.name in names]
        self.net = nw.EncodedNetwork(self.params, self.ctx, ps, rounds)
        self.n, self.L = 1 << ps.log_n, ps.n_data
        dev = f"cuda:{device}"
        self.stream = torch.cuda.current_stream(device)
        self.d_ins, self.d_outs, self.sps, self.sos, self.k_ins, self.caps = [], [], [], [], [], []
        for r, info in enumerate(self.net.infos):
            first, last = self.net.rounds[r].name == "stem", self.net.rounds[r].name == "fc"
            x = np.random.default_rng(seed + 100 + r).uniform(0.0, 1.0, info["E_in"])
            sp = None if first else sf.sf_permutation(seed + 4, r, info["E_in"])
            so = None if last else sf.sf_permutation(seed + 4, r + 1, info["E_out"])
            xs = x if sp is None else x[sp.astype(np.int64)]
            d_in = torch.empty((info["k_in"], 2, self.L, self.n), dtype=torch.int64, device=dev)
            sf.sf_encrypt(self.ctx, self.sk, sf.sf_encode_input(xs, ps.delta), seed + 1000 + r, d_in, info["k_in"])
            self.d_ins.append(d_in)
            self.d_outs.append(torch.empty((info["n_groups"], 2, self.L, self.n), dtype=torch.int64, device=dev))
            self.sps.append(sp)
            self.sos.append(so)
            self.k_ins.append(info["k_in"])
            self.caps.append(info["n_groups"])
        self.layer_of = list(range(len(self.net.rounds)))   # input slot -> round
        self.x_seed_of = [seed + 100 + r for r in range(len(self.net.rounds))]   # input slot -> input seed
        self.ct_bytes = 2 * self.L * self.n * 8

    def add_requests(self, r: int, copies: int):
        """copies more encrypted inputs of round r, as if from other requests
        (fresh inputs and encryption seeds under the same client key); their
        slots are appended to the round lists (weights shared with round r)."""
        sf, torch = self.sf, self.torch
        info = self.net.infos[r]
        for c in range(copies):
            x_seed = self._seed + 7000 + 31 * r + c
            self.x_seed_of.append(x_seed)
            x = np.random.default_rng(x_seed).uniform(0.0, 1.0, info["E_in"])
            sp = self.sps[r]
            xs = x if sp is None else x[sp.astype(np.int64)]
            d_in = torch.empty_like(self.d_ins[r])
            sf.sf_encrypt(self.ctx, self.sk, sf.sf_encode_input(xs, self.ps.delta), self._seed + 9000 + c, d_in,
                          info["k_in"])
            self.d_ins.append(d_in)
            self.d_outs.append(torch.empty_like(self.d_outs[r]))
            self.sps.append(sp)
            self.sos.append(self.sos[r])
            self.k_ins.append(info["k_in"])
            self.caps.append(info["n_groups"])
            self.layer_of.append(r)

    def per_layer(self, r: int):
        self.sf.sf_eval_linear_layer(self.ctx, self.net.layers[self.layer_of[r]], self.rk, self.d_ins[r], self.k_ins[r],
                                     self.sps[r], self.sos[r], self.d_outs[r], self.caps[r], self.stream)

    def batched(self, idx=None):
        idx = list(range(len(self.d_ins))) if idx is None else idx
        return self.sf.sf_eval_layers(self.ctx, [self.net.layers[self.layer_of[r]] for r in idx], [self.rk] * len(idx),
                                      [self.d_ins[r] for r in idx], [self.k_ins[r] for r in idx],
                                      [self.sps[r] for r in idx], [self.sos[r] for r in idx],
                                      [self.d_outs[r] for r in idx], [self.caps[r] for r in idx], self.stream)

    def autotune(self, idx):
        return self.sf.sf_autotune_layers(self.ctx, [self.net.layers[r] for r in idx], [self.rk] * len(idx),
                                          [self.d_ins[r] for r in idx], [self.k_ins[r] for r in idx],
                                          [self.sps[r] for r in idx], [self.sos[r] for r in idx],
                                          [self.d_outs[r] for r in idx], [self.caps[r] for r in idx], 1, self.stream)

    def destroy(self):
        sf = self.sf
        self.net.destroy()
        sf.sf_rotkeys_destroy(self.rk)
        sf.sf_secret_key_destroy(self.sk)
        sf.sf_ctx_destroy(self.ctx)
        sf.sf_params_destroy(self.params)
        self.d_ins = self.d_outs = []

    def max_err(self, slots) -> float:
        """Max |decoded - float64| over every output of the given input slots."""
        from paper_2509_01253_gb300 import network as nw
        sf = self.sf
        worst = 0.0
        for k in slots:
            r = self.layer_of[k]
            info = self.net.infos[r]
            res = np.zeros((info["n_groups"], self.L, self.n), dtype=np.uint64)
            sf.sf_decrypt(self.ctx, self.sk, self.d_outs[k], info["n_groups"], res, self.stream)
            vals = nw.decode_outputs(self.net, r, res)
            x = np.random.default_rng(self.x_seed_of[k]).uniform(0.0, 1.0, info["E_in"])
            ref = nw.round_float_reference(self.net, r, x)
            if self.sos[k] is not None:
                ref = ref[self.sos[k].astype(np.int64)]
            worst = max(worst, float(np.abs(vals - ref).max()))
        return worst


def timed(torch, stream, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_network(args, local: int) -> int:
    """One JSON line: the network's rounds as one batched sf_eval_layers call
    (after autotuning the key-switch batch on the three smallest rounds) and
    as one sf_eval_linear_layer call per round, with per-round times."""
    import torch
    torch.cuda.set_device(local)
    seed = 300 if args.workload == "resnet18" else 400
    nw_ = NetworkWorkload(args.workload, local, seed)
    nw_._seed = seed
    for kv in args.ctx_opt:
        name, val = kv.split("=", 1)
        nw_.sf.sf_ctx_set_option(nw_.ctx, name, int(val))
    torch_ = torch
    sf = nw_.sf
    R = len(nw_.net.rounds)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")
    clocks = ClockSampler(local)
    clocks.start()
    if args.layer_stats:
        g = RingShape(sf.sf_params_get_info(nw_.params))
        out = {"workload": args.workload, "n": nw_.n, "L": nw_.L, "layer_stats": {}}
        names = [r.name for r in nw_.net.rounds]
        for name in args.layer_stats.split(","):
            r = names.index(name)
            timed(torch_, nw_.stream, lambda: nw_.per_layer(r))
            sf.sf_kernel_stats_reset(nw_.ctx)
            sf.sf_ctx_set_option(nw_.ctx, "kernel_timing", 1)
            flush_l2(flush)
            t = timed(torch_, nw_.stream, lambda: nw_.per_layer(r))
            sf.sf_ctx_set_option(nw_.ctx, "kernel_timing", 0)
            ks = launches(sf, nw_.ctx)
            tot = sum(ms for _, ms in ks.values())
            info = nw_.net.infos[r]
            out["layer_stats"][name] = {
                "info": info, "ms_instrumented": t,
                "kernels": {k: {"launches": c, "ms": m} for k, (c, m) in ks.items() if c},
                "roofline": roofline_of(ks, 1, g, info, tot, {"sm_mhz": None})}
        out["clocks"] = clocks.stop()
        print(json.dumps(out), flush=True)
        return 0
    rec = {"metric": METRIC, "unit": UNIT, "workload": args.workload, "rounds": R,
           "ks_total": nw_.net.total_ks(), "outputs_total": sum(i["E_out"] for i in nw_.net.infos),
           "n": nw_.n, "L": nw_.L, "data": "synthetic: per-round inputs U(0,1), Kaiming-uniform weights"}
    # one call per round (each round captured in its own graph on first use)
    per_round = [0.0] * R
    for rep in range(2):           # 0: warm-up (captures), 1: timed
        for r in range(R):
            flush_l2(flush)
            t = timed(torch_, nw_.stream, lambda: nw_.per_layer(r))
            if rep == 1:
                per_round[r] = t
    rec["per_layer_ms"] = {nw_.net.rounds[r].name: per_round[r] for r in range(R)}
    rec["per_layer_form"] = {"total_ms": sum(per_round), "layers_per_s": R / (sum(per_round) / 1e3),
                             "ks_batch": "default"}
    err = nw_.max_err(range(R)) if args.workload == "resnet18" else nw_.max_err([R - 1, R - 2])
    # autotune the launch batch on the smallest rounds, then the whole network as one batch
    small = sorted(range(R), key=lambda r: nw_.net.infos[r]["E_out"])[:3]
    best, best_ms = nw_.autotune(small)
    rec["autotune"] = {"rounds": [nw_.net.rounds[r].name for r in small], "ks_batch": best, "ms": best_ms}
    flush_l2(flush)
    timed(torch_, nw_.stream, nw_.batched)        # capture + run
    t_b = []
    for _ in range(max(1, min(args.steps, 2))):
        flush_l2(flush)
        t_b.append(timed(torch_, nw_.stream, nw_.batched))
    tb = min(t_b)
    rec["batched_form"] = {"total_ms": tb, "layers_per_s": R / (tb / 1e3), "ks_batch": best,
                           "calls": 1, "timed_runs": len(t_b)}
    err_b = nw_.max_err(range(R)) if args.workload == "resnet18" else nw_.max_err([R - 1, R - 2])
    rec["value"] = R / (tb / 1e3)
    rec["speedup_batched_vs_per_layer"] = sum(per_round) / tb
    rec["max_abs_err"] = {"per_layer": err, "batched": err_b,
                          "rounds_checked": "all" if args.workload == "resnet18" else "last two"}
    rec["clocks"] = clocks.stop()
    print(json.dumps(rec), flush=True)
    return 0


def run_request_e2e(args, local: int) -> int:
    """One encrypted inference request end to end: every round on the
    device (one engine call each, rotation keys and weights resident) with
    the simulated client between rounds (decrypt, ReLU, re-encode, encrypt).
    Reports per-round device time, the request's wall time and the max error
    of every round against float64 on the client's actual round input."""
    import torch
    import paper_2509_01253_gb300 as sf
    from paper_2509_01253_gb300 import network as nw
    from paper_2509_01253_gb300 import workloads as wl
    torch.cuda.set_device(local)
    kind = args.workload
    ps = wl.PARAMS[NET_PARAMS[kind]]
    params = sf.sf_params_create(ps.log_n, ps.n_data, ps.data_bits, ps.n_special, ps.special_bits, ps.sigma)
    ctx = sf.sf_ctx_create(params, local)
    sk = sf.sf_keygen(ctx, 401)
    rk = sf.sf_gen_rotation_keys(ctx, sk, None, 405)
    net = nw.EncodedNetwork(params, ctx, ps, wl.resnet_rounds(kind), gamma=args.gamma)
    calib = None
    if args.gamma_plan:
        # a gamma = 0 request of another image with the per-round kernel split
        split = []
        c_cal = nw.ClientState(net, wl.network_input(kind, 412), session_seed=414, request_seed=413)
        net.gammas = [0] * len(net.rounds)
        ms_cal = nw.run_request(net, sk, rk, c_cal, split=split)
        net.gammas = nw.plan_gammas(net, split)
        calib = {"what": "gamma = 0 request of another image, kernel timing on (no graph replay)",
                 "per_layer_ms": {net.rounds[r].name: ms_cal[r] for r in range(len(ms_cal))},
                 "leaf_ms": {net.rounds[r].name: split[r][0] for r in range(len(split))},
                 "kernel_ms": {net.rounds[r].name: split[r][1] for r in range(len(split))},
                 "device_total_s": sum(ms_cal) / 1e3}
    x = wl.network_input(kind, 402)
    client = nw.ClientState(net, x, session_seed=404, request_seed=403)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    from paper_2509_01253_gb300 import protocol
    log = protocol.CommLog()
    t0 = time.perf_counter()
    ms = nw.run_request(net, sk, rk, client, keep_trace=True, log=log)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    errs = []
    for r, (x_in, y) in enumerate(client.trace):
        errs.append(float(np.abs(y - nw.round_float_reference(net, r, x_in)).max()))
    R = len(net.rounds)
    rec = {"metric": METRIC, "unit": UNIT, "workload": kind,
           "gamma": "per-round plan" if args.gamma_plan else args.gamma, "rounds": R, "n": 1 << ps.log_n,
           "L": ps.n_data,
           "ks_total": net.total_ks(), "outputs_total": sum(i["E_out"] for i in net.infos),
           "data": "synthetic: image U(0,1), Kaiming-uniform weights, pool folded into the first block",
           "per_layer_ms": {net.rounds[r].name: ms[r] for r in range(R)},
           "device_total_s": sum(ms) / 1e3, "request_wall_s": wall,
           "layers_per_s_device": R / (sum(ms) / 1e3), "value": R / wall,
           "max_abs_err_per_round": errs, "max_abs_err": max(errs), "clocks": clk,
           "protocol": log.summary(),
           "note": "each round's first call includes its graph capture"}
    if calib is not None:
        rec["gamma_per_round"] = {net.rounds[r].name: net.gammas[r] for r in range(R)}
        rec["calibration"] = calib
    print(json.dumps(rec), flush=True)
    return 0


def conv16_record(local: int, steps: int = 5) -> dict:
    """The conv16 round (N = 2^14, 3 x 50-bit + 1): autotuned, warmed up, then
    `steps` timed rounds with the L2 flushed between them, and its decryption
    check; the kernel with the largest device time from an instrumented pass."""
    import torch
    wl_ = Workload(local, "conv16")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")
    wl_.step()
    tuned = wl_.autotune()
    for _ in range(3):
        wl_.step()
    ms = []
    for _ in range(steps):
        flush_l2(flush)
        ms.append(timed(torch, wl_.stream, wl_.step))
    err = wl_.check()
    sf = wl_.sf
    sf.sf_kernel_stats_reset(wl_.ctx)
    sf.sf_ctx_set_option(wl_.ctx, "kernel_timing", 1)
    for _ in range(2):
        flush_l2(flush)
        wl_.step()
    torch.cuda.synchronize()
    ks = launches(sf, wl_.ctx)
    sf.sf_ctx_set_option(wl_.ctx, "kernel_timing", 0)
    g = RingShape(sf.sf_params_get_info(wl_.params))
    tot = sum(m for _, m in ks.values())
    top = roofline_of(ks, 2, g, wl_.info, tot, {"sm_mhz": None}, sm_count=sm_count_of(local))
    wl_.destroy()
    t = sum(ms) / len(ms)
    return {"workload": LAYERS["conv16"][3], "value": 1e3 / t, "unit": UNIT, "ms_per_step": t, "step_ms": ms,
            "steps": steps, "autotuned": tuned, "max_abs_err": err,
            "top_kernel": {k: top[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac",
                                              "share_of_device_time")},
            "kernels": {k: {"launches_per_layer": c // 2, "ms_per_layer": m / 2} for k, (c, m) in ks.items() if c}}


def gamma2_record(local: int, kind: str = "r34", steps: int = 3) -> dict:
    """The same layer at partial trace extraction level gamma = 2 (Sec. 4.3,
    4.4, Lemma 1 at t = 2): the client also uploads RLWE(m(X^3)) per input
    ciphertext, the leaves read twice the ciphertexts and the packing skips
    the tau_3 level.  Time per layer (L2 flushed between steps) against the
    gamma = 0 layer, key switches, upload bytes, and the decryption check
    (packed values halved)."""
    import torch
    wl_ = Workload(local, kind)
    sf = wl_.sf
    from paper_2509_01253_gb300 import workloads as wlm
    d_pow = torch.zeros_like(wl_.d_in)
    sf.sf_encrypt(wl_.ctx, wl_.sk, sf.sf_client_power(wl_.params, wl_.msg, wl_.k_in, 3), 7404, d_pow, wl_.k_in)
    case = wl_.case

    def step2():
        sf.sf_eval_linear_layer_gamma(wl_.ctx, wl_.layer, wl_.rk, 2, wl_.d_in, d_pow, wl_.k_in, case.sigma_prev,
                                      case.sigma_out, wl_.d_out, wl_.G, wl_.stream)

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")
    out = {}
    for name, fn in (("gamma0", wl_.step), ("gamma2", step2)):
        fn()
        for _ in range(2):
            fn()
        ms = []
        for _ in range(steps):
            flush_l2(flush)
            ms.append(timed(torch, wl_.stream, fn))
        out[name] = {"ms_per_layer": sum(ms) / len(ms), "step_ms": ms}
    sf.sf_sync(wl_.ctx, wl_.stream)
    res = np.zeros((wl_.G, wl_.L, wl_.n), dtype=np.uint64)
    sf.sf_decrypt(wl_.ctx, wl_.sk, wl_.d_out, wl_.G, res, wl_.stream)
    vals = sf.sf_decode(wl_.params, res, wl_.G, wl_.n // wl_.info["group_size"], wl_.info["E_out"],
                        2 * wl_.ps.delta ** 2)
    ref = wlm.float_reference(case)
    if case.sigma_out is not None:
        ref = ref[case.sigma_out.astype(np.int64)]
    n, G = wl_.info["group_size"], wl_.G
    ks2 = G * (n // 2 - 1 + (wl_.n.bit_length() - 1) - (n.bit_length() - 1))
    rec = {"workload": wl_.desc, "key_switches": {"gamma0": wl_.info["ks_count"], "gamma2": ks2},
           "upload_bytes": {"gamma0": wl_.k_in * wl_.ct_bytes, "gamma2": 2 * wl_.k_in * wl_.ct_bytes},
           "max_abs_err_gamma2": float(np.abs(vals - ref).max()),
           "speedup_gamma2_vs_gamma0": out["gamma0"]["ms_per_layer"] / out["gamma2"]["ms_per_layer"], **out}
    wl_.destroy()
    return rec


def serving_record(local: int, rate: float = 0.3, duration: float = 30.0, drain: float = 60.0) -> dict:
    """Continuous-batching server below capacity: ResNet-20 requests at
    N = 2^14 from 4 client keys, Poisson arrivals at `rate` per second for
    `duration` seconds; p50/p99 latency of the completed requests (each
    checked against the float64 network), and one request alone."""
    from paper_2509_01253_gb300 import serve
    from paper_2509_01253_gb300 import workloads as wl
    pool = serve.Pool(wl.PARAMS["conv16"], ["resnet20"], 4, local, key_seed=7000, priority=-1)
    budget = 48 << 30
    srv = serve.Server({"c2": pool}, {"resnet20": "c2"}, budget, max_active=1, max_batch=1)
    alone = serve.run_arrivals(srv, [(0.0, "resnet20", 0, 99)], drain=600.0)
    arr = serve.poisson_arrivals(rate, duration, {"resnet20": 1.0}, 4, seed=31)
    srv = serve.Server({"c2": pool}, {"resnet20": "c2"}, budget, max_active=16)
    st = serve.run_arrivals(srv, arr, drain, verify=True)
    pool.destroy()
    return {"what": f"ResNet-20 (3x32x32, 20 rounds, N = 2^14) requests, Poisson {rate} req/s for {duration:.0f} s, "
                    f"4 client keys, continuous batching; latency = arrival to logits, client steps included",
            "rate_req_s": rate, "p50_latency_s": st["p50_latency_s"], "p99_latency_s": st["p99_latency_s"],
            "arrivals": st["arrivals"], "completed": st["completed"], "rejected": st["rejected"],
            "served_layers_per_s": st["layers_per_s"], "mean_rounds_per_call": st["mean_rounds_per_call"],
            "max_abs_err_vs_float64": st["max_abs_err_vs_float64"],
            "alone_latency_s": alone["p50_latency_s"]}


BATCH_ROUNDS = ["s3b0c1", "s3b0c2", "s3b1c1", "s3b1c2", "fc"]


def batched_record(local: int, kind: str, names: list, copies: int = 0, reps: int = 2) -> dict:
    """Rounds of a network (`names`, each with its own encrypted input, plus
    `copies` more inputs of the first named round, as from concurrent
    requests): one sf_eval_layers call against one sf_eval_linear_layer call
    per round (both captured once, L2 flushed before each timed run, best of
    `reps`), with the decryption check of every output of both forms."""
    import torch
    seed = {"resnet18": 300, "resnet20": 500}[kind]
    nw_ = NetworkWorkload(kind, local, seed, names=names)
    nw_._seed = seed
    if copies:
        nw_.add_requests(0, copies)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")
    S = len(nw_.d_ins)

    def per_layer_all():
        for k in range(S):
            nw_.per_layer(k)

    per_layer_all()
    t_p = []
    for _ in range(reps):
        flush_l2(flush)
        t_p.append(timed(torch, nw_.stream, per_layer_all))
    err_p = nw_.max_err(range(S))
    nw_.batched()
    t_b = []
    for _ in range(reps):
        flush_l2(flush)
        t_b.append(timed(torch, nw_.stream, nw_.batched))
    err_b = nw_.max_err(range(S))
    ks = sum(nw_.net.infos[r]["ks_count"] for r in nw_.layer_of)
    n_ring = nw_.n
    nw_.destroy()
    what = f"{kind} rounds {', '.join(names)} at N = {n_ring}"
    if copies:
        what += f", the first round for {copies + 1} concurrent requests"
    return {"what": what + "; each input its own synthetic encryption; default launch batch",
            "round_evaluations": S, "key_switches": ks, "per_layer_ms": min(t_p), "batched_ms": min(t_b),
            "speedup_batched_vs_per_layer": min(t_p) / min(t_b), "layers_per_s_batched": S / (min(t_b) / 1e3),
            "layers_per_s_per_layer": S / (min(t_p) / 1e3), "max_abs_err": {"per_layer": err_p, "batched": err_b}}


R20_LATE = ["s2b0c1", "s2b0c2", "s2b1c1", "s2b1c2", "s2b2c1", "s2b2c2", "fc"]


def sm_count_of(local: int) -> int:
    import torch
    return torch.cuda.get_device_properties(local).multi_processor_count


def main():
    args = parse()
    dist, ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, dist, ws, rank)
    if args.workload == "resnet34" and not args.layer_stats:
        return run_request_e2e(args, local) if rank == 0 else 0
    if args.workload in ("resnet18", "resnet34"):
        return run_network(args, local) if rank == 0 else 0
    if args.workload == "serve":
        from paper_2509_01253_gb300 import serve
        return serve.bench(args, local) if rank == 0 else 0
    import torch
    import paper_2509_01253_gb300 as sf
    torch.cuda.set_device(local)
    n_sm = sm_count_of(local)
    wl_ = Workload(local, args.workload, small=args.small)
    for kv in args.ctx_opt:
        name, val = kv.split("=", 1)
        sf.sf_ctx_set_option(wl_.ctx, name, int(val))
    stream = wl_.stream
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")
    # one round, its decryption check (it may grow the context's workspace,
    # which drops captured graphs) and the autotuner, then the warm-up proper
    wl_.step()
    torch.cuda.synchronize()
    err = wl_.check()
    tuned = None if args.no_autotune else wl_.autotune()
    for _ in range(max(3, args.warmup)):
        wl_.step()
    torch.cuda.synchronize()
    # ---- timed region: device-resident inputs
    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
    sf.sf_kernel_stats_reset(wl_.ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    for i in range(args.steps):
        flush_l2(flush)
        ev[i][0].record(stream)
        wl_.step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    # the decryption check again, on the output of the last timed step (the
    # autotuned configuration), outside the timed region
    err_final = wl_.check()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    stats = launches(sf, wl_.ctx)
    n_launch = sum(c for c, _ in stats.values())
    total_s = max_over_ranks(dist, total_s)
    value = replicas_value(ws, args.steps, total_s)
    # ---- end to end: host buffers through the C ABI, copies inside the timed region
    e2e_steps = max(1, min(args.steps, 5))
    pin_in = torch.empty((wl_.k_in, 2, wl_.L, wl_.n), dtype=torch.int64, pin_memory=True)
    pin_in.copy_(wl_.d_in.cpu())
    pin_out = torch.empty((wl_.G, 2, wl_.L, wl_.n), dtype=torch.int64, pin_memory=True)
    h_in = pin_in.numpy().view(np.uint64)
    h_out = pin_out.numpy().view(np.uint64)
    for _ in range(2):
        sf.sf_eval_linear_layer_host(wl_.ctx, wl_.layer, wl_.rk, h_in, wl_.k_in, wl_.case.sigma_prev,
                                     wl_.case.sigma_out, h_out, wl_.G, stream)
    if dist:
        dist.barrier()
    e2e_s = 0.0
    for i in range(e2e_steps):
        flush_l2(flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sf.sf_eval_linear_layer_host(wl_.ctx, wl_.layer, wl_.rk, h_in, wl_.k_in, wl_.case.sigma_prev,
                                     wl_.case.sigma_out, h_out, wl_.G, stream)
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(dist, e2e_s)
    e2e_value = replicas_value(ws, e2e_steps, e2e_s)
    h2d = wl_.k_in * wl_.ct_bytes + 4 * (wl_.info["E_in"] + wl_.info["E_out"])
    d2h = wl_.G * wl_.ct_bytes
    # ---- per-kernel device time (instrumented pass: events around every launch)
    sf.sf_kernel_stats_reset(wl_.ctx)
    sf.sf_ctx_set_option(wl_.ctx, "kernel_timing", 1)
    k_steps = max(2, min(args.steps, 3))
    for _ in range(k_steps):
        flush_l2(flush)
        wl_.step()
    torch.cuda.synchronize()
    kstats = launches(sf, wl_.ctx)
    sf.sf_ctx_set_option(wl_.ctx, "kernel_timing", 0)
    total_kernel_ms = sum(ms for _, ms in kstats.values())
    p_info = sf.sf_params_get_info(wl_.params)
    probe = measure_probe(sf, wl_.ctx)
    roofline = roofline_of(kstats, k_steps, RingShape(p_info), wl_.info, total_kernel_ms, clk, probe=probe,
                           sm_count=n_sm)
    ntt = ntt_record(sf, torch, wl_, p_info, probe, flush)
    kernel_table = {k: {"launches_per_layer": c // k_steps, "ms_per_layer": m / k_steps} for k, (c, m) in kstats.items() if c}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": wl_.desc, "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "autotuned": tuned, "ctx_options": args.ctx_opt, "max_abs_err": err,
                       "max_abs_err_final": err_final, "e2e_steps": e2e_steps},
            "clocks": clk, "gpu_launches": n_launch // 1, "step_ms": step_ms,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": roofline, "ntt": ntt, "probe": probe, "kernels": kernel_table}
    wl_.destroy()
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu_baseline:
        v, cores, desc = oracle_sample(args.workload if not args.small else args.workload)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0 and args.workload == "r34" and not args.no_extras and not args.small:
        extras = {}
        for name, fn in (("conv16", lambda: conv16_record(local)), ("gamma2", lambda: gamma2_record(local)),
                         ("serving", lambda: serving_record(local)),
                         ("batched_vs_per_layer", lambda: batched_record(local, "resnet18", BATCH_ROUNDS)),
                         ("batched_small_rounds", lambda: batched_record(local, "resnet20", R20_LATE)),
                         ("batched_requests", lambda: batched_record(local, "resnet20", ["s2b1c1"], copies=7)),
                         ("pp_ntt", lambda: pp_ntt_record(local, flush)),
                         ("torus_ks", lambda: tq_record(local, flush))):
            t0 = time.perf_counter()
            try:
                extras[name] = fn()
            except Exception as exc:    # a sub-record must not lose the main line
                extras[name] = {"error": f"{type(exc).__name__}: {exc}"}
            extras[name]["wall_s"] = time.perf_counter() - t0
            torch.cuda.empty_cache()
        line.update(extras)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
