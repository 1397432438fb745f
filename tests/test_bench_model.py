"""The bench's work model (host logic, no GPU): per-kernel operation counts
against closed forms of the key switch at the benchmark ring, and the
probe-weighted arithmetic ceiling."""
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
