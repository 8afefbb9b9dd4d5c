"""Measured pipe peaks and the look-back scan with its bounded wait.

The roofline of the blending (Sec. 3.1 Eqns. 1-2, Alg. 1) divides by the
FP32, SFU and ALU issue rates that seele_measure_peaks measures; they must
agree with the device's SM count and lane counts at a plausible clock.  The
look-back scan behind the no-alloc sort is checked against numpy, and its
bounded wait is made to run out on purpose (one block withholds its sums, the
wait limit is short): the call must report a timeout, every block before the
withheld one must still be right, and the next ordinary call must succeed.
Nothing faults or hangs: every wait is bounded and the withholding block
still finishes.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def seele():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_05168_gb300 as p
    return p


def test_measured_peaks_match_the_device(seele):
    import torch
    props = torch.cuda.get_device_properties(0)
    p = seele.measure_peaks(0)
    assert p["sm_count"] == props.multi_processor_count
    ghz = p["sm_clock_max_mhz"] / 1000.0
    assert ghz > 0.5
    # lanes per SM per clock: 128 FP32 (FMA); ex2 16 or (GB300) 32; the ALU
    # pipe 64 (float min/max and integer logic alike)
    for key, lanes, lo, hi in (("fp32_tops", 128, 0.5, 1.1), ("sfu_tops", 16, 0.5, 2.2),
                               ("alu_fmnmx_tops", 64, 0.5, 1.1), ("alu_lop3_tops", 64, 0.5, 1.1)):
        nominal = p["sm_count"] * lanes * ghz / 1000.0
        assert lo * nominal <= p[key] <= hi * nominal, (key, p[key], nominal)


def _wrapped_exclusive_sum(x):
    c = np.cumsum(x.astype(np.uint64)) & np.uint64(0xFFFFFFFF)
    return np.concatenate([[0], c[:-1]]).astype(np.uint32)


@pytest.mark.parametrize("n", [1, 4096, 16 * 4096 + 123, 300_001])
def test_exclusive_scan_matches_numpy(seele, n):
    import torch
    rs = np.random.default_rng(n)
    x = rs.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    t = torch.from_numpy(x.view(np.int32)).cuda()
    for _ in range(2):
        st, out = seele.exclusive_scan(t)
        assert st == 0
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), _wrapped_exclusive_sum(x))


def test_bounded_wait_gives_up_and_the_next_call_succeeds(seele):
    import torch
    n = 16 * 4096
    x = np.arange(n, dtype=np.uint32) % 7
    t = torch.from_numpy(x.view(np.int32)).cuda()
    exp = _wrapped_exclusive_sum(x)
    st, out = seele.exclusive_scan(t, withhold_block=5, spin_limit=2000)
    assert st == 5  # SEELE_ERR_TIMEOUT
    got = out.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got[:5 * 4096], exp[:5 * 4096])   # before the withheld block
    st, out = seele.exclusive_scan(t)
    assert st == 0
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), exp)
