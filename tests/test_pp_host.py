"""Host side of the prime-power ring entry points (no GPU): parameter checks
return SF_EINVAL before any device work, and without a CUDA device a valid
ring fails with SF_ECUDA (no CPU fallback)."""
import pytest

import paper_2509_01253_gb300 as sf


@pytest.mark.parametrize("t,alpha,L,bits", [(2, 5, 1, 50), (9, 2, 1, 50), (11, 2, 1, 50), (3, 1, 1, 50),
                                            (3, 8, 1, 50), (3, 3, 0, 50), (3, 3, 13, 50), (3, 3, 1, 62),
                                            (3, 3, 1, 19)])
def test_pp_ring_parameter_checks(t, alpha, L, bits):
    with pytest.raises(sf.SafhireError) as e:
        sf.sf_pp_ring_create(t, alpha, L, bits, 0)
    assert e.value.status == sf.SF_EINVAL


def test_pp_ring_needs_a_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(sf.SafhireError) as e:
        sf.sf_pp_ring_create(3, 7, 2, 50, 0)
    assert e.value.status == sf.SF_ECUDA


@pytest.mark.parametrize("t,alpha,D,l", [(3, 3, 1, 3), (3, 3, 65537, 1), (3, 3, 512, 0), (3, 3, 512, 9),
                                         (3, 3, 2 ** 16, 4), (3, 3, 3, 34), (2, 5, 512, 3), (3, 8, 512, 3)])
def test_tq_ring_parameter_checks(t, alpha, D, l):
    """Torus rings: the gadget limits (2 <= D <= 65536, 1 <= l <= 8, D^l <= 2^53)
    and the ring limits are checked before any device work."""
    with pytest.raises(sf.SafhireError) as e:
        sf.sf_tq_ring_create(t, alpha, D, l, 0)
    assert e.value.status == sf.SF_EINVAL


def test_tq_ring_needs_a_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(sf.SafhireError) as e:
        sf.sf_tq_ring_create(5, 5, 310, 5, 0)
    assert e.value.status == sf.SF_ECUDA


def test_tq_calls_reject_a_null_ring():
    """Every torus call checks its ring and buffers before any device work."""
    for call in (lambda: sf.sf_tq_ring_info(None),
                 lambda: sf.sf_tq_decompose(None, 8, 8, 1),
                 lambda: sf.sf_tq_encrypt(None, 8, 8, 8, 8, 8, 1),
                 lambda: sf.sf_tq_decrypt(None, 8, 8, 8, 1),
                 lambda: sf.sf_tq_ksk(None, 8, 2, 8, 8, 8),
                 lambda: sf.sf_tq_key_prepare(None, 8, 8, 8),
                 lambda: sf.sf_tq_keyswitch(None, 8, 16, 1, 2, 8),
                 lambda: sf.sf_tq_hom_trace(None, 8, 16, 1, 0, {})):
        with pytest.raises(sf.SafhireError) as e:
            call()
        assert e.value.status == sf.SF_EINVAL
    sf.sf_tq_ring_destroy(None)   # a null ring is ignored
