"""The bench's work model (host logic, no GPU): per-kernel operation counts
against closed forms of the key switch at the benchmark ring, and the
probe-weighted arithmetic ceiling."""
import pytest

import bench


def _ring(n, L, K):
    return bench.RingShape({"n": n, "n_data": L, "n_special": K, "dnum": -(-L // K)})


def test_key_switch_butterflies_are_twenty_limb_transforms():
    # N = 2^14, 3 data + 1 special: ModUp inverse 3, extensions 9, ModDown 2 + 6 = 20 limb NTTs
    g = _ring(1 << 14, 3, 1)
    per_ntt = (g.n // 2) * 14
    ks = ["ks1_inv_row", "ks2_modup_col", "ks3_inner_row", "ks3_inv_row_p", "ks4_moddown_col", "ks5_finish_row"]
    bfly = sum(bench.kernel_ops(k, g)[0] + bench.kernel_ops(k, g)[1] for k in ks)
    assert bfly == 20 * per_ntt
    # key multiply-accumulates: 2 parts x dnum digits x (L + K) moduli x N
    assert bench.kernel_ops("ks3_inner_row", g)[2] == 2 * 3 * 4 * g.n
    # one-limb digits convert with no product; two-limb digits do
    assert bench.kernel_ops("ks2_modup_col", g)[2] == 3 * g.n
    g2 = _ring(1 << 15, 4, 2)
    assert bench.kernel_ops("ks2_modup_col", g2)[2] == 4 * g2.n + 2 * (2 * 4) * g2.n


def test_work_totals_and_probe_ceiling():
    g = _ring(1 << 14, 3, 1)
    probe = {"fwd_bfly": 1000.0, "inv_bfly": 800.0, "mac": 1100.0}
    for k in ["ks_gather", "ks2_modup_col", "ks3_inner_row", "ks4_moddown_col", "leaf_row"]:
        nbytes, mm = bench.kernel_work(k, g)
        ops = bench.kernel_ops(k, g)
        assert mm == sum(ops) and nbytes > 0
        c = bench.probe_ceiling(ops, probe)
        assert 800.0 <= c <= 1100.0
    assert bench.probe_ceiling(bench.kernel_ops("ks1_inv_row", g), probe) == 800.0
    assert bench.probe_ceiling((0, 0, 0), probe) is None
    assert bench.kernel_work("no_such_kernel", g) is None


def test_roofline_record_arithmetic():
    """roofline_of on synthetic per-kernel statistics: the top kernel by device
    time, achieved = algorithmic work x items / time per layer, the derived and
    measured ceilings, and DRAM traffic scaled to one launch."""
    g = _ring(1 << 14, 3, 1)
    info = {"k_in": 1, "ks_count": 16384, "E_out": 16384}
    k_steps = 10
    kstats = {"ks3_inner_row": (15 * k_steps, 250.0), "ks2_modup_col": (15 * k_steps, 170.0),
              "elementwise": (k_steps, 999.0)}          # no work model: never the top kernel
    probe = {"fwd_bfly": 1000.0, "inv_bfly": 800.0, "mac": 1100.0}
    rec = bench.roofline_of(kstats, k_steps, g, info, 420.0, {"sm_mhz": 2070.0}, probe=probe)
    assert rec["kernel"] == "ks3_inner_row" and rec["bound"] == "alu"
    per_layer_s = 250.0 / k_steps / 1e3
    nbytes, mm = bench.kernel_work("ks3_inner_row", g)
    assert rec["achieved"] == pytest.approx(mm * 16384 / per_layer_s / 1e9)
    assert rec["peak"] == pytest.approx(bench.alu_peak(152, 2070.0) / 1e9)
    assert rec["frac"] == pytest.approx(rec["achieved"] / rec["peak"])
    assert rec["hbm_view"]["achieved"] == pytest.approx(nbytes * 16384 / per_layer_s / 1e9)
    ceil = bench.probe_ceiling(bench.kernel_ops("ks3_inner_row", g), probe)
    assert rec["alu_view"]["probe_peak"] == pytest.approx(ceil)
    assert rec["alu_view"]["frac_of_probe"] == pytest.approx(rec["achieved"] / ceil)
    assert rec["launches_per_layer"] == 15
    assert rec["traffic"] is None                      # no capture of this kernel at this ring
    assert rec["share_of_device_time"] == pytest.approx(250.0 / 420.0)
    # traffic scales a per-item capture to a launch; the SM count sets the derived peak
    bench.TRAFFIC_PER_ITEM[("ks3_inner_row", 14)] = 2.5e6
    try:
        rec2 = bench.roofline_of(kstats, k_steps, g, info, 420.0, {"sm_mhz": 2070.0}, probe=probe, sm_count=148)
    finally:
        del bench.TRAFFIC_PER_ITEM[("ks3_inner_row", 14)]
    assert rec2["traffic"] == pytest.approx(2.5e6 * 16384 / 15)
    assert rec2["peak"] == pytest.approx(148 * 64 * 2070e6 / 10 / 1e9)
    assert "148 SMs" in rec2["peak_source"]
