"""Host logic of the per-round extraction level (Sec. 4.3, 4.4): key-switch
counts per round and level, and the planner's choice from a gamma = 0
kernel split.  No GPU."""
from paper_2509_01253_gb300 import network as nw


class _Net:
    """The parts of an EncodedNetwork the planner reads."""
    ks_count = nw.EncodedNetwork.ks_count

    def __init__(self, infos):
        self.infos = infos
        self.rounds = list(range(len(infos)))
        self.gammas = [0] * len(infos)


def _info(n_groups, group_size, ks):
    return {"n_groups": n_groups, "group_size": group_size, "ks_count": ks}


def test_ks_count_per_level():
    # N = 2^14, groups of 8 outputs: 7 merges + log2(2^14 / 8) = 11 trace steps each
    net = _Net([_info(2, 8, 2 * (7 + 11)), _info(1, 1, 14), _info(3, 2, 3 * (1 + 13))])
    assert [net.ks_count(r, 0) for r in range(3)] == [36, 14, 42]
    # gamma = 2 drops the n/2 merges of the tau_3 level per group, or one trace step when n = 1
    assert [net.ks_count(r, 2) for r in range(3)] == [36 - 2 * 4, 14 - 1, 42 - 3 * 1]
    net.gammas = [2, 0, 2]
    assert [net.ks_count(r) for r in range(3)] == [28, 14, 39]


def test_plan_from_kernel_split():
    # ks halves at gamma = 2 in round 0 (16 -> 8), and in round 1 (2 -> 1)
    net = _Net([_info(1, 16, 16), _info(1, 2, 2)])
    assert net.ks_count(0, 2) == 8 and net.ks_count(1, 2) == 1
    # leaves exactly doubling (leaf_factor 2): leaf 1 of 3 ms predicts 2 + 2 / 2 = 3,
    # not below 0.98 x 3 -> gamma 0; leaf 0.5 of 3 ms predicts 1 + 2.5 / 2 = 2.25 -> gamma 2
    assert nw.plan_gammas(net, [(1.0, 3.0), (1.0, 3.0)], leaf_factor=2.0) == [0, 0]
    assert nw.plan_gammas(net, [(0.5, 3.0), (2.0, 3.0)], leaf_factor=2.0) == [2, 0]
    # exactly at break-even: gamma 0
    assert nw.plan_gammas(net, [(1.0, 3.0), (0.0, 1.0)], margin=0.0, leaf_factor=2.0) == [0, 2]
    # the default leaf factor 2.2: leaf 0.85 of 2.94 ms predicts 1.87 + 2.09 / 2 = 2.915, below
    # 2.94 but not below 0.98 x 2.94 = 2.881: the margin keeps a near break-even round at 0
    assert nw.plan_gammas(net, [(0.85, 2.94), (0.0, 1.0)], margin=0.0) == [2, 2]
    assert nw.plan_gammas(net, [(0.85, 2.94), (0.0, 1.0)]) == [0, 2]
    # a round that gains with leaves doubling but not at 2.2: leaf 1.2 of 4 ms
    # predicts 2.4 + 1.4 = 3.8 (gamma 2) at factor 2, 2.64 + 1.4 = 4.04 (gamma 0) at 2.2
    assert nw.plan_gammas(net, [(1.2, 4.0), (1.0, 1.0)], leaf_factor=2.0) == [2, 0]
    assert nw.plan_gammas(net, [(1.2, 4.0), (1.0, 1.0)]) == [0, 0]
